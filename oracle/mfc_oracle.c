/*
 * FP64 oracle for the coupled flow + advection-diffusion lattice Boltzmann solvers of
 * Tsompanas et al., "Modelling Microbial Fuel Cells using lattice Boltzmann methods"
 * (arXiv 1802.07525), Sec. 3.1.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU restatement of
 * the method, used to check the CUDA path.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never links, calls or falls
 * back to it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, round to nearest).
 * A second, timing-only build adds -fopenmp: the two node loops of a step then share their
 * rows among the host cores.  Every node's arithmetic is the same in both builds (each node is
 * written by one thread, from the previous step's values), so their results are identical; the
 * plain build is the one the tests check against.
 *
 * Conventions (readings of the paper where it is silent or garbled are listed at each place):
 *   - lattice units dx = dt = 1, rho0 = 1;
 *   - node index k = x + nx*(y + ny*z) (x fastest);
 *   - populations are SoA: f[i*N + k];
 *   - the flow axis is x in 2-D and z in 3-D; the inlet is at the low end of that axis;
 *   - node classes are bit flags: 1 = blocked for the flow lattice, 2 = blocked for the
 *     transport lattice, 4 = consumption (sink) node.
 *
 * Parity status: every function here is pinned by the "not gpu" tests (closed forms,
 * conservation laws, symmetry, published generator vectors); none is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

enum { BC_WALL = 0, BC_PERIODIC = 1, BC_INOUT = 2 };
enum { CLS_FLOW_SOLID = 1, CLS_ADE_SOLID = 2, CLS_SINK = 4 };
enum { SRC_NODE = 0, SRC_BOUNCE = 1, SRC_INLET = 2, SRC_OUTLET = 3 };

typedef struct {
    int dim;           /* 2 or 3 */
    int nx, ny, nz;    /* nz = 1 in 2-D */
    int bc[3];         /* per axis: BC_WALL, BC_PERIODIC, BC_INOUT (flow axis only) */
    int ade_q;         /* 5 (D2Q5), 7 (D3Q7) or 9 (D2Q9 with the Eq. 5 equilibrium) */
    int ade_outlet;    /* 0 zero-gradient, 1 Dirichlet at c_out */
    double tau;        /* flow relaxation time, Eq. 4 */
    double tau_c;      /* transport relaxation time tau_D, Eq. 12 */
    double u_in;       /* inlet speed along the flow axis */
    double rho_in;     /* density of the moving wall that forms the flow inlet */
    double rho_out;    /* outlet density (pressure reference) */
    double c_in;       /* inlet concentration (Dirichlet input) */
    double c_out;      /* outlet concentration when ade_outlet = 1 */
    double k_sink;     /* first-order consumption rate on sink nodes */
    double u_scale;    /* factor applied to the flow velocity seen by the transport solver */
    double k_half;     /* half-saturation concentration K_s of the substrate factor of Eq. 16;
                          0 = the first-order limit k*C */
} orc_params;

/* Consumption on a sink node at concentration C (Eq. 16, substrate factor): the saturating
 * rate q_max C / (C + K_s) with q_max = k_sink K_s, so that k_sink is the rate per unit
 * concentration at low C; K_s = 0 selects the first-order limit k_sink C.  The mediator factor
 * M_ox / (M_ox + K_Mox) is taken as constant and folded into k_sink. */
static double consumption(const orc_params *p, double C)
{
    if (p->k_half > 0.0) return p->k_sink * p->k_half * C / (p->k_half + C);
    return p->k_sink * C;
}

/* ------------------------------------------------------------------------------------------
 * Velocity sets.
 * D2Q9 follows Eqs. 1-3 with weights Eqs. 6-8.  The order of c5..c8 is fixed by the pairs of
 * Eq. 11 (south wall: 5<->7, 2<->4, 6<->8), i.e. 5=(1,1), 6=(-1,1), 7=(-1,-1), 8=(1,-1).
 * D3Q19 (flow, 3-D) and D2Q5 / D3Q7 (transport) are the standard sets; the paper only states
 * that the 3-D extension is direct (Sec. 2) and gives no ordering, so opposites are adjacent.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int q;
    const int (*c)[3];
    const int *opp;
    const double *w;
    double cs2;
} vset;

static const int D2Q9_C[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const int D2Q9_OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double D2Q9_W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int D2Q5_C[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}};
static const int D2Q5_OPP[5] = {0, 3, 4, 1, 2};
static const double D2Q5_W[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};

static const int D3Q19_C[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const int D3Q19_OPP[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
static const double D3Q19_W[19] = {
    1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int D3Q7_C[7][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                                 {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const int D3Q7_OPP[7] = {0, 2, 1, 4, 3, 6, 5};
static const double D3Q7_W[7] = {1.0 / 4.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0,
                                 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0};

static vset flow_set(const orc_params *p)
{
    vset v;
    if (p->dim == 2) {
        v.q = 9; v.c = D2Q9_C; v.opp = D2Q9_OPP; v.w = D2Q9_W;
    } else {
        v.q = 19; v.c = D3Q19_C; v.opp = D3Q19_OPP; v.w = D3Q19_W;
    }
    v.cs2 = 1.0 / 3.0;
    return v;
}

static vset ade_set(const orc_params *p)
{
    vset v;
    if (p->ade_q == 9) {
        v.q = 9; v.c = D2Q9_C; v.opp = D2Q9_OPP; v.w = D2Q9_W; v.cs2 = 1.0 / 3.0;
    } else if (p->ade_q == 7) {
        v.q = 7; v.c = D3Q7_C; v.opp = D3Q7_OPP; v.w = D3Q7_W; v.cs2 = 1.0 / 4.0;
    } else {
        v.q = 5; v.c = D2Q5_C; v.opp = D2Q5_OPP; v.w = D2Q5_W; v.cs2 = 1.0 / 3.0;
    }
    return v;
}

static long n_nodes(const orc_params *p) { return (long)p->nx * p->ny * p->nz; }
static int flow_axis(const orc_params *p) { return p->dim == 2 ? 0 : 2; }

/* ------------------------------------------------------------------------------------------
 * Equilibria.
 * Flow, Eq. 5: F_i^(0) = w_i rho [1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u].  The printed
 * c = dx/(dt sqrt 3) would make the coefficients 9, 81/2, 9/2; the reading taken is the
 * standard one (c = dx/dt = 1, sound speed squared 1/3), which Table 1 confirms: tau_D =
 * 0.5036 and D = 0.0012 mm^2/s satisfy D = (tau_D - 1/2)/3 exactly.
 * Transport, Eq. 12: on D2Q5 / D3Q7 the equilibrium is the linear one,
 * G_i^(0) = w_i C (1 + c_i.u / cs2); on D2Q9 (ade_q = 9) it is Eq. 5 reused with C in
 * place of rho, as the text after Eq. 12 says.
 * ------------------------------------------------------------------------------------------ */
static void flow_equilibrium(const vset *v, double rho, const double u[3], double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < v->q; ++i) {
        double cu = v->c[i][0] * u[0] + v->c[i][1] * u[1] + v->c[i][2] * u[2];
        feq[i] = v->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

static void ade_equilibrium(const vset *v, double conc, const double u[3], double *geq)
{
    if (v->q == 9) {
        flow_equilibrium(v, conc, u, geq);
        return;
    }
    for (int i = 0; i < v->q; ++i) {
        double cu = v->c[i][0] * u[0] + v->c[i][1] * u[1] + v->c[i][2] * u[2];
        geq[i] = v->w[i] * conc * (1.0 + cu / v->cs2);
    }
}

ORC_API void orc_flow_equilibrium(int dim, double rho, const double *u, double *feq)
{
    orc_params p;
    memset(&p, 0, sizeof p);
    p.dim = dim;
    vset v = flow_set(&p);
    double uu[3] = {u[0], u[1], dim == 3 ? u[2] : 0.0};
    flow_equilibrium(&v, rho, uu, feq);
}

ORC_API void orc_ade_equilibrium(int ade_q, double conc, const double *u, double *geq)
{
    orc_params p;
    memset(&p, 0, sizeof p);
    p.ade_q = ade_q;
    vset v = ade_set(&p);
    double uu[3] = {u[0], u[1], ade_q == 7 ? u[2] : 0.0};
    ade_equilibrium(&v, conc, uu, geq);
}

/* Velocity-set tables, for the isotropy pins. */
ORC_API int orc_velocity_set(int which, int *c, int *opp, double *w)
{
    orc_params p;
    memset(&p, 0, sizeof p);
    vset v;
    if (which == 9) { p.dim = 2; v = flow_set(&p); }
    else if (which == 19) { p.dim = 3; v = flow_set(&p); }
    else { p.ade_q = which; v = ade_set(&p); }
    for (int i = 0; i < v.q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = v.c[i][a];
        opp[i] = v.opp[i];
        w[i] = v.w[i];
    }
    return v.q;
}

/* ------------------------------------------------------------------------------------------
 * Pull streaming with boundaries (Eq. 4 streaming part, Eq. 11 bounce-back).
 * The population that arrives at x along c_i comes from s = x - c_i.
 *   - s outside the lattice across a wall, or s blocked: half-way bounce-back, i.e. the
 *     population that left x along the opposite direction returns (Eq. 11; the wall sits
 *     half-way along the link, so a channel of NY nodes has width NY).
 *   - s before the inlet (flow axis): SRC_INLET.  Flow: bounce-back from a wall moving at
 *     the inlet velocity.  Transport: an equilibrium ghost at the inlet concentration.
 *   - s past the outlet: SRC_OUTLET, with *src = s moved back onto the last layer (unless
 *     that node is blocked, which gives bounce-back).  Flow: equilibrium ghost at the
 *     outlet density with the velocity of that last-layer node (zero velocity gradient,
 *     pressure reference).  Transport: a copy of that node's population (zero gradient), or
 *     an equilibrium ghost at c_out when the outlet is Dirichlet.
 * Precedence: wall or solid first, then inlet, then outlet.  Blocked nodes hold no
 * populations and are not collided.
 * ------------------------------------------------------------------------------------------ */
static int pull_source(const orc_params *p, const uint8_t *cls, int blocked_bit, int x, int y,
                       int z, const int c[3], long *src)
{
    int n[3] = {p->nx, p->ny, p->nz};
    int s[3] = {x - c[0], y - c[1], z - c[2]};
    int fa = flow_axis(p);
    int inlet = 0, outlet = 0;
    for (int a = 0; a < 3; ++a) {
        if (s[a] >= 0 && s[a] < n[a]) continue;
        if (p->bc[a] == BC_PERIODIC) {
            s[a] = (s[a] + n[a]) % n[a];
        } else if (p->bc[a] == BC_INOUT && a == fa) {
            if (s[a] < 0) inlet = 1; else outlet = 1;
        } else {
            return SRC_BOUNCE; /* a wall (an inlet/outlet on a cross axis is treated as a wall) */
        }
    }
    if (inlet) return SRC_INLET;
    if (outlet) s[fa] = n[fa] - 1;
    long j = s[0] + (long)n[0] * (s[1] + (long)n[1] * s[2]);
    if (cls[j] & blocked_bit) return SRC_BOUNCE;
    *src = j;
    return outlet ? SRC_OUTLET : SRC_NODE;
}

/* Flow outlet ghost: F_i^(0)(rho_out, u) with u the velocity of the post-collision
 * populations at last-layer node s (collision conserves mass and momentum, so this is the
 * velocity of that node's streamed populations of the previous step). */
static double outlet_equilibrium(const vset *v, const orc_params *p, const double *f, long N,
                                 long s, int i)
{
    double r = 0.0, j[3] = {0, 0, 0};
    for (int m = 0; m < v->q; ++m) {
        r += f[m * N + s];
        for (int a = 0; a < 3; ++a) j[a] += v->c[m][a] * f[m * N + s];
    }
    double u[3] = {j[0] / r, j[1] / r, j[2] / r};
    double feq[19];
    flow_equilibrium(v, p->rho_out, u, feq);
    return feq[i];
}

/* One flow step (Eq. 4 with Eq. 5, moments Eqs. 9-10, bounce-back Eq. 11).
 * In:  f   = post-collision populations of the previous step.
 * Out: fn  = post-collision populations of this step (0 on blocked nodes);
 *      rho, u = moments of the streamed populations (before collision), 0 on blocked nodes. */
ORC_API void orc_flow_step(const orc_params *p, const uint8_t *cls, const double *f, double *fn,
                           double *rho, double *u)
{
    vset v = flow_set(p);
    long N = n_nodes(p);
    int fa = flow_axis(p);
    double uin[3] = {0, 0, 0};
    uin[fa] = p->u_in;
    /* inlet: bounce-back from a wall moving at u_in (momentum-corrected bounce-back),
     * F_i = F*_opp(i) + 2 w_i rho_in (c_i . u_in) / cs2, which injects exactly rho_in*u_in
     * per unit of inlet cross-section */
    double bb_in[19];
    for (int i = 0; i < v.q; ++i) {
        double cu = v.c[i][0] * uin[0] + v.c[i][1] * uin[1] + v.c[i][2] * uin[2];
        bb_in[i] = 2.0 * v.w[i] * p->rho_in * cu / v.cs2;
    }

#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = x + (long)p->nx * (y + (long)p->ny * z);
                if (cls[k] & CLS_FLOW_SOLID) {
                    for (int i = 0; i < v.q; ++i) fn[i * N + k] = 0.0;
                    rho[k] = 0.0;
                    for (int a = 0; a < p->dim; ++a) u[a * N + k] = 0.0;
                    continue;
                }
                double fin[19];
                for (int i = 0; i < v.q; ++i) {
                    long s;
                    switch (pull_source(p, cls, CLS_FLOW_SOLID, x, y, z, v.c[i], &s)) {
                    case SRC_NODE: fin[i] = f[i * N + s]; break;
                    case SRC_BOUNCE: fin[i] = f[v.opp[i] * N + k]; break;
                    case SRC_INLET: fin[i] = f[v.opp[i] * N + k] + bb_in[i]; break;
                    default: fin[i] = outlet_equilibrium(&v, p, f, N, s, i); break;
                    }
                }
                double r = 0.0, j[3] = {0, 0, 0};
                for (int i = 0; i < v.q; ++i) {
                    r += fin[i];
                    for (int a = 0; a < 3; ++a) j[a] += v.c[i][a] * fin[i];
                }
                double uu[3] = {j[0] / r, j[1] / r, j[2] / r};
                double feq[19];
                flow_equilibrium(&v, r, uu, feq);
                for (int i = 0; i < v.q; ++i) fn[i * N + k] = fin[i] - (fin[i] - feq[i]) / p->tau;
                rho[k] = r;
                for (int a = 0; a < p->dim; ++a) u[a * N + k] = uu[a];
            }
}

/* One transport step (Eq. 12 with the consumption sink, concentration Eq. 13).
 * The velocity u (dim x N) is held fixed during the transport solve (text after Eq. 12); it
 * is scaled by u_scale and taken as zero on nodes blocked for the flow (biofilm is
 * impermeable to flow, Sec. 3.3, but still takes part in transport).
 * Consumption: the rate of consumption() on sink nodes (first order k*C, or the saturating
 * substrate factor of Eq. 16), removed in proportion to the weights, so that sum_i G_i loses
 * exactly that rate per sink node per step.  Eq. 12 prints no source term.
 * Out: gn (0 on blocked nodes) and conc = moment of the streamed populations (Eq. 13). */
ORC_API void orc_ade_step(const orc_params *p, const uint8_t *cls, const double *g, double *gn,
                          const double *u, double *conc)
{
    vset v = ade_set(p);
    long N = n_nodes(p);
    int fa = flow_axis(p);
    double uin[3] = {0, 0, 0};
    uin[fa] = p->u_in;
    double geq_in[19], geq_out[19];
    ade_equilibrium(&v, p->c_in, uin, geq_in);
    ade_equilibrium(&v, p->c_out, uin, geq_out);

#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = x + (long)p->nx * (y + (long)p->ny * z);
                if (cls[k] & CLS_ADE_SOLID) {
                    for (int i = 0; i < v.q; ++i) gn[i * N + k] = 0.0;
                    conc[k] = 0.0;
                    continue;
                }
                double uk[3] = {0, 0, 0};
                if (!(cls[k] & CLS_FLOW_SOLID))
                    for (int a = 0; a < p->dim; ++a) uk[a] = u[a * N + k] * p->u_scale;
                double gin[19];
                for (int i = 0; i < v.q; ++i) {
                    long s;
                    switch (pull_source(p, cls, CLS_ADE_SOLID, x, y, z, v.c[i], &s)) {
                    case SRC_NODE: gin[i] = g[i * N + s]; break;
                    case SRC_BOUNCE: gin[i] = g[v.opp[i] * N + k]; break;
                    case SRC_INLET: gin[i] = geq_in[i]; break;
                    default: gin[i] = p->ade_outlet == 1 ? geq_out[i] : g[i * N + s]; break;
                    }
                }
                double C = 0.0;
                for (int i = 0; i < v.q; ++i) C += gin[i];
                double geq[19];
                ade_equilibrium(&v, C, uk, geq);
                double sink = (cls[k] & CLS_SINK) ? consumption(p, C) : 0.0;
                for (int i = 0; i < v.q; ++i)
                    gn[i * N + k] = gin[i] - (gin[i] - geq[i]) / p->tau_c - v.w[i] * sink;
                conc[k] = C;
            }
}

/* Global sums used by the steady-state test and the current (FP64).
 * out[0] = sum |u - u_prev|^2, out[1] = sum |u|^2, out[2] = sum rho      (flow-active nodes)
 * out[3] = sum (C - C_prev)^2, out[4] = sum C^2,  out[5] = sum C        (transport-active)
 * out[6] = sum over sink nodes of the consumption (the substrate uptake that sets the current,
 *          Eqs. 16, 20)
 * out[7] = number of non-finite values met
 * out[8] = number of flow-active nodes outside the range of the scheme: |u|^2 >= cs^2 = 1/3
 *          (at or above the lattice sound speed, where the low-Mach expansion behind Eq. 5 no
 *          longer holds) or rho <= 0.  A solver guard: the paper states no such limit.  (A
 *          density bound would be wrong: the 128x64 channel's steady state, behind its nearly
 *          impermeable porous block, has rho close to 2 upstream.) */
ORC_API void orc_sums(const orc_params *p, const uint8_t *cls, const double *rho, const double *u,
                      const double *u_prev, const double *conc, const double *conc_prev,
                      double *out)
{
    long N = n_nodes(p);
    for (int m = 0; m < 9; ++m) out[m] = 0.0;
    for (long k = 0; k < N; ++k) {
        if (!(cls[k] & CLS_FLOW_SOLID) && rho) {
            double speed2 = 0.0;
            for (int a = 0; a < p->dim; ++a) {
                double d = u[a * N + k] - u_prev[a * N + k];
                out[0] += d * d;
                out[1] += u[a * N + k] * u[a * N + k];
                speed2 += u[a * N + k] * u[a * N + k];
                if (!isfinite(u[a * N + k])) out[7] += 1.0;
            }
            out[2] += rho[k];
            if (!isfinite(rho[k])) out[7] += 1.0;
            if (speed2 >= 1.0 / 3.0 || rho[k] <= 0.0) out[8] += 1.0;
        }
        if (!(cls[k] & CLS_ADE_SOLID) && conc) {
            double d = conc[k] - conc_prev[k];
            out[3] += d * d;
            out[4] += conc[k] * conc[k];
            out[5] += conc[k];
            if (cls[k] & CLS_SINK) out[6] += consumption(p, conc[k]);
            if (!isfinite(conc[k])) out[7] += 1.0;
        }
    }
}

static double rel_residual(double d2, double n2)
{
    if (n2 > 0.0) return sqrt(d2 / n2);
    return d2 > 0.0 ? INFINITY : 0.0;
}

/* Initial state (the paper is silent): flow at rest, F_i = w_i on open nodes; no substrate,
 * G_i = 0 everywhere. */
ORC_API void orc_init_state(const orc_params *p, const uint8_t *cls, double *f, double *g)
{
    vset vf = flow_set(p), va = ade_set(p);
    long N = n_nodes(p);
    for (long k = 0; k < N; ++k) {
        for (int i = 0; i < vf.q; ++i) f[i * N + k] = (cls[k] & CLS_FLOW_SOLID) ? 0.0 : vf.w[i];
        for (int i = 0; i < va.q; ++i) g[i * N + k] = 0.0;
    }
}

enum { MODE_SEQUENTIAL = 0, MODE_CONCURRENT = 1 };

typedef struct {
    long steps_flow, steps_ade;
    double res_flow, res_ade, current, mass, substrate;
    int converged;
    int unstable;  /* stopped at a check that found a node outside the range (out[8] of orc_sums) */
} orc_result;

/* Iterate to equilibrium (method steps 2 and 3 of Sec. 3; "enough time steps until an
 * equilibrium is reached", Sec. 4, which fixes no criterion).  The test is the mean relative
 * change per step since the previous check,
 *     r = ||v^n - v^m|| / ((n - m) ||v^n||) < tol,
 * evaluated at the check steps n: the multiples of check_every and the last step allowed;
 * m is the previous check step, or the step of the fields given on entry (the last step run
 * before the call).  With check_every = 1 it is the per-step change ||v^n - v^(n-1)|| / ||v^n||.
 * A check that finds a flow node outside the scheme's range (out[8] of orc_sums) ends the solve
 * there, not converged, with res->unstable set.
 * SEQUENTIAL: the flow runs to equilibrium, then transport runs with that velocity frozen
 * (the paper's order).  CONCURRENT: both advance together, transport using the same step's
 * flow velocity; both residuals must fall below their tolerances.
 * f, g: state in/out.  rho, u, conc: fields of the last step, in/out.  Returns converged. */
ORC_API int orc_solve_steady(const orc_params *p, const uint8_t *cls, double *f, double *g,
                             double *rho, double *u, double *conc, int mode, double tol_flow,
                             double tol_ade, long max_steps, int check_every, orc_result *res)
{
    vset vf = flow_set(p), va = ade_set(p);
    long N = n_nodes(p);
    int d = p->dim;
    double *f2 = calloc((size_t)vf.q * N, sizeof(double));
    double *g2 = calloc((size_t)va.q * N, sizeof(double));
    double *u_prev = calloc((size_t)d * N, sizeof(double));   /* fields at the previous check */
    double *c_prev = calloc((size_t)N, sizeof(double));
    double s[9];
    memset(res, 0, sizeof *res);
    int conv_f = 0, conv_a = 0;
    if (check_every < 1) check_every = 1;
    memcpy(u_prev, u, sizeof(double) * d * N);
    memcpy(c_prev, conc, sizeof(double) * N);

    if (mode == MODE_SEQUENTIAL) {
        long m = 0;
        for (long n = 1; n <= max_steps; ++n) {
            orc_flow_step(p, cls, f, f2, rho, u);
            memcpy(f, f2, sizeof(double) * vf.q * N);
            res->steps_flow = n;
            if (n % check_every == 0 || n == max_steps) {
                orc_sums(p, cls, rho, u, u_prev, NULL, NULL, s);
                res->res_flow = rel_residual(s[0], s[1]) / (double)(n - m);
                res->mass = s[2];
                memcpy(u_prev, u, sizeof(double) * d * N);
                m = n;
                if (s[8] > 0.0) { res->unstable = 1; break; }
                if (res->res_flow < tol_flow) { conv_f = 1; break; }
            }
        }
        m = 0;
        for (long n = 1; n <= max_steps && !res->unstable; ++n) {
            orc_ade_step(p, cls, g, g2, u, conc);
            memcpy(g, g2, sizeof(double) * va.q * N);
            res->steps_ade = n;
            if (n % check_every == 0 || n == max_steps) {
                orc_sums(p, cls, NULL, u, u, conc, c_prev, s);
                res->res_ade = rel_residual(s[3], s[4]) / (double)(n - m);
                res->substrate = s[5];
                res->current = s[6];
                memcpy(c_prev, conc, sizeof(double) * N);
                m = n;
                if (res->res_ade < tol_ade) { conv_a = 1; break; }
            }
        }
    } else {
        long m = 0;
        for (long n = 1; n <= max_steps; ++n) {
            orc_flow_step(p, cls, f, f2, rho, u);
            orc_ade_step(p, cls, g, g2, u, conc);
            memcpy(f, f2, sizeof(double) * vf.q * N);
            memcpy(g, g2, sizeof(double) * va.q * N);
            res->steps_flow = res->steps_ade = n;
            if (n % check_every == 0 || n == max_steps) {
                orc_sums(p, cls, rho, u, u_prev, conc, c_prev, s);
                res->res_flow = rel_residual(s[0], s[1]) / (double)(n - m);
                res->res_ade = rel_residual(s[3], s[4]) / (double)(n - m);
                res->mass = s[2];
                res->substrate = s[5];
                res->current = s[6];
                memcpy(u_prev, u, sizeof(double) * d * N);
                memcpy(c_prev, conc, sizeof(double) * N);
                m = n;
                if (s[8] > 0.0) { res->unstable = 1; break; }
                if (res->res_flow < tol_flow && res->res_ade < tol_ade) {
                    conv_f = conv_a = 1;
                    break;
                }
            }
        }
    }
    res->converged = conv_f && conv_a;
    free(f2); free(g2); free(u_prev); free(c_prev);
    return res->converged;
}

/* ------------------------------------------------------------------------------------------
 * Biofilm growth rule of the 2048x1024 cycle workload (a simplified stand-in for the agent
 * model of Sec. 3.3): an open node (no class bit set) becomes biofilm when one of its
 * flow-lattice neighbours is a consumption node, its concentration is above c_thresh
 * (strictly), and a uniform draw is below prob.  New biofilm is impermeable to flow and
 * consumes substrate (Sec. 3.3: "the updated biofilm as impermeable"), i.e. class
 * CLS_FLOW_SOLID | CLS_SINK.  All decisions read the classes from before the pass.
 * Neighbours are the non-rest directions of the flow velocity set, inside the lattice only.
 * Draw: h = splitmix64(seed ^ (cycle << 32) ^ k); convert when (h >> 11) < prob * 2^53.
 * splitmix64 is Steele, Lea and Flood's generator (OOPSLA 2014) as published by Vigna:
 * z = x + 0x9e3779b97f4a7c15; z = (z ^ z>>30) * 0xbf58476d1ce4e5b9;
 * z = (z ^ z>>27) * 0x94d049bb133111eb; return z ^ z>>31.
 * Returns the number of converted nodes.
 * ------------------------------------------------------------------------------------------ */
ORC_API uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

ORC_API long orc_biofilm_convert(const orc_params *p, const uint8_t *cls, const double *conc,
                                 uint64_t seed, uint64_t cycle, double prob, double c_thresh,
                                 uint8_t *cls_out)
{
    vset v = flow_set(p);
    long N = n_nodes(p);
    double lim = floor(prob * 9007199254740992.0); /* prob * 2^53 */
    long count = 0;
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = x + (long)p->nx * (y + (long)p->ny * z);
                cls_out[k] = cls[k];
                if (cls[k] != 0) continue;
                int near = 0;
                for (int i = 1; i < v.q && !near; ++i) {
                    int sx = x + v.c[i][0], sy = y + v.c[i][1], sz = z + v.c[i][2];
                    if (sx < 0 || sx >= p->nx || sy < 0 || sy >= p->ny || sz < 0 || sz >= p->nz)
                        continue;
                    long j = sx + (long)p->nx * (sy + (long)p->ny * sz);
                    if (cls[j] & CLS_SINK) near = 1;
                }
                if (!near || !(conc[k] > c_thresh)) continue;
                uint64_t h = orc_splitmix64(seed ^ (cycle << 32) ^ (uint64_t)k);
                if ((double)(h >> 11) < lim) {
                    cls_out[k] = CLS_FLOW_SOLID | CLS_SINK;
                    ++count;
                }
            }
    return count;
}

/* ------------------------------------------------------------------------------------------
 * Agent-based biofilm formation, Sec. 3.3: attachment, growth and spreading of biomass, once
 * per model iteration (between steady solves).  Per node: C^bio (bio[k], mg biomass / L).
 * Readings where the section leaves a choice:
 *   - the front is the set of open nodes (no class bit) without biomass that have an electrode
 *     node (blocked for both lattices) among their flow-lattice neighbours;
 *   - attachment: the k_ata front nodes with the smallest keys are set to C_0^bio, where the key
 *     of node k is (the top 32 bits of h) << 32 | k with
 *     h = splitmix64(splitmix64(seed ^ ATTACH_TAG) ^ (cycle << 32) ^ k); all front nodes when
 *     there are fewer (keys are unique, so the choice is exact);
 *   - growth follows the double Monod law of Eq. 16 with the mediator factor, a biomass yield and
 *     the time span folded into one parameter mu: on every transport-open node with biomass,
 *     C^bio <- C^bio (1 + mu s), s = C+ / (C+ + K_s), C+ = max(C, 0), C the local substrate
 *     concentration of the last solve; attachment comes first, so new cells grow too;
 *   - spreading: the nodes with C^bio > C_max^bio when spreading starts (not electrode) are
 *     taken in increasing node order; one still above C_max^bio when reached spreads.  Free
 *     cells are open nodes without biomass inside the lattice.  If a neighbour is free, the
 *     receiving cell is a random one of its free neighbours (in direction order); otherwise a
 *     random walk starts at the node: each step draws one of the Q - 1 directions, a step onto
 *     the electrode or out of the lattice is lost, a step onto a cell already on the walk's path
 *     erases the loop back to it (loop-erased walk), and the walk ends on the first free cell.
 *     Every cell with biomass on the path then passes its biomass one cell further along the
 *     path towards the free cell, which frees the first cell of the path; that cell receives
 *     fr_spr C^bio of the spreading node, which keeps the rest.  A walk that has taken max_walk
 *     steps without reaching a free cell gives up (no change);
 *   - draws of the spreading pass: the n-th draw of the pass is
 *     splitmix64(splitmix64(seed ^ SPREAD_TAG ^ (cycle << 32)) ^ n), n = 0, 1, ...; a choice
 *     among m options takes (draw >> 32) % m;
 *   - afterwards every non-electrode node with biomass is biofilm: impermeable to the flow and
 *     consuming substrate (class 5; Sec. 3.3 and the conclusions); other classes are kept.
 * stats: [0] attached, [1] front nodes, [2] spreading events, [3] walks given up,
 *        [4] walk steps taken, [5] nodes with biomass, [6] total biomass (sum of C^bio).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t seed;
    int k_ata;
    double C0_bio, Cmax_bio, fr_spr, mu, K_s;
    int max_walk;
} orc_agent;

#define ORC_ATTACH_TAG 0x6174746163680000ULL /* "attach" */
#define ORC_SPREAD_TAG 0x7370726561640000ULL /* "spread" */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int inside(const orc_params *p, int x, int y, int z)
{
    return x >= 0 && x < p->nx && y >= 0 && y < p->ny && z >= 0 && z < p->nz;
}

ORC_API void orc_agent_step(const orc_params *p, const uint8_t *cls, const double *conc,
                            const orc_agent *a, uint64_t cycle, double *bio, uint8_t *cls_out,
                            double *stats)
{
    vset v = flow_set(p);
    long N = n_nodes(p);
    const uint8_t ELECTRODE = CLS_FLOW_SOLID | CLS_ADE_SOLID;
    for (int m = 0; m < 7; ++m) stats[m] = 0.0;

    /* attachment */
    uint64_t *keys = malloc(sizeof(uint64_t) * (size_t)(N > 0 ? N : 1));
    long nf = 0;
    uint64_t base = orc_splitmix64(a->seed ^ ORC_ATTACH_TAG);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long k = x + (long)p->nx * (y + (long)p->ny * z);
                if (cls[k] != 0 || bio[k] != 0.0) continue;
                int front = 0;
                for (int i = 1; i < v.q; ++i) {
                    int sx = x + v.c[i][0], sy = y + v.c[i][1], sz = z + v.c[i][2];
                    if (!inside(p, sx, sy, sz)) continue;
                    if ((cls[sx + (long)p->nx * (sy + (long)p->ny * sz)] & ELECTRODE) == ELECTRODE) front = 1;
                }
                if (!front) continue;
                uint64_t h = orc_splitmix64(base ^ (cycle << 32) ^ (uint64_t)k);
                keys[nf++] = ((h >> 32) << 32) | (uint64_t)(uint32_t)k;
            }
    qsort(keys, (size_t)nf, sizeof(uint64_t), cmp_u64);
    long na = nf < a->k_ata ? nf : a->k_ata;
    for (long j = 0; j < na; ++j) bio[(long)(uint32_t)keys[j]] = a->C0_bio;
    stats[0] = (double)na;
    stats[1] = (double)nf;
    free(keys);

    /* growth (double Monod, Eq. 16) */
    for (long k = 0; k < N; ++k) {
        if (bio[k] > 0.0 && !(cls[k] & CLS_ADE_SOLID)) {
            double C = conc[k] > 0.0 ? conc[k] : 0.0;
            bio[k] = bio[k] * (1.0 + a->mu * (C / (C + a->K_s)));
        }
    }

    /* spreading */
    long *list = malloc(sizeof(long) * (size_t)(N > 0 ? N : 1));
    long nl = 0;
    for (long k = 0; k < N; ++k)
        if (bio[k] > a->Cmax_bio && !(cls[k] & CLS_ADE_SOLID)) list[nl++] = k;
    long *path = malloc(sizeof(long) * ((size_t)a->max_walk + 2));
    uint64_t sbase = orc_splitmix64(a->seed ^ ORC_SPREAD_TAG ^ (cycle << 32));
    uint64_t ndraw = 0;
    for (long e = 0; e < nl; ++e) {
        long k = list[e];
        if (!(bio[k] > a->Cmax_bio)) continue;
        int x = (int)(k % p->nx), y = (int)((k / p->nx) % p->ny), z = (int)(k / ((long)p->nx * p->ny));
        /* free neighbours, in direction order */
        long freen[19];
        int nfree = 0;
        for (int i = 1; i < v.q; ++i) {
            int sx = x + v.c[i][0], sy = y + v.c[i][1], sz = z + v.c[i][2];
            if (!inside(p, sx, sy, sz)) continue;
            long j = sx + (long)p->nx * (sy + (long)p->ny * sz);
            if (!(cls[j] & ELECTRODE) && bio[j] == 0.0) freen[nfree++] = j;
        }
        long target;
        if (nfree > 0) {
            uint64_t d = orc_splitmix64(sbase ^ ndraw++);
            target = freen[(d >> 32) % (uint64_t)nfree];
        } else {
            /* loop-erased random walk from k to the first free cell */
            long len = 1;
            path[0] = k;
            int found = 0;
            for (int step = 0; step < a->max_walk && !found; ++step) {
                stats[4] += 1.0;
                uint64_t d = orc_splitmix64(sbase ^ ndraw++);
                int i = 1 + (int)((d >> 32) % (uint64_t)(v.q - 1));
                long cur = path[len - 1];
                int cx = (int)(cur % p->nx), cy = (int)((cur / p->nx) % p->ny);
                int cz = (int)(cur / ((long)p->nx * p->ny));
                int sx = cx + v.c[i][0], sy = cy + v.c[i][1], sz = cz + v.c[i][2];
                if (!inside(p, sx, sy, sz)) continue;
                long j = sx + (long)p->nx * (sy + (long)p->ny * sz);
                if (cls[j] & CLS_ADE_SOLID) continue; /* electrode: the step is lost */
                long at = -1;
                for (long m = 0; m < len; ++m)
                    if (path[m] == j) { at = m; break; }
                if (at >= 0) { len = at + 1; continue; } /* erase the loop */
                path[len++] = j;
                if (bio[j] == 0.0) found = 1;
            }
            if (!found) { stats[3] += 1.0; continue; }
            /* shove: every cell with biomass passes it one cell on, from the free end back */
            for (long m = len - 1; m >= 2; --m) bio[path[m]] = bio[path[m - 1]];
            target = path[1];
            bio[target] = 0.0;
        }
        double t = a->fr_spr * bio[k];
        bio[k] = bio[k] - t;
        bio[target] = t;
        stats[2] += 1.0;
    }
    free(path);
    free(list);

    /* classes: biomass makes biofilm (impermeable to flow, consuming) */
    for (long k = 0; k < N; ++k) {
        cls_out[k] = cls[k];
        if (bio[k] > 0.0 && !(cls[k] & CLS_ADE_SOLID)) cls_out[k] = CLS_FLOW_SOLID | CLS_SINK;
        if (bio[k] > 0.0) stats[5] += 1.0;
        stats[6] += bio[k];
    }
}

ORC_API int orc_agent_size(void) { return (int)sizeof(orc_agent); }

/* ------------------------------------------------------------------------------------------
 * Bio-electrochemical model of the anode, Sec. 3.2, Eqs. 14-21, lumped over the anode.
 * Units: M_ox, M_red, M_total in mg mediator / mg biomass; q_max in mg substrate /
 * (mg biomass day); I in A; E_0, overpotentials and voltages in V; resistances in ohm; A_a in
 * m^2; I_0 in A/m^2; V_a in L; C^bio in mg biomass / L; gamma in mg / mol; dt in s.
 * Readings (the paper gives the equations but not their time base or every constant):
 *   - Eq. 15 is an explicit step of dt seconds: the consumption term Y q_a is per day, so it is
 *     divided by 86400; the current term gamma I / (m F V_a C^bio) is per second;
 *   - C_s / (C_s + K_s) in Eq. 16 is the mean substrate factor over the biofilm, S, from the
 *     lattice solve;
 *   - I in Eq. 20 is implicit (n_act of Eq. 19 depends on I); it is found here as the root of
 *     g(I) = I - (E_0 - n_conc - n_act(I)) / (R_int + R_ext) * M_red / (eps + M_red)
 *     by bisection, re-evaluating Eq. 19 at every trial I;
 *   - the voltage across the load is V = I R_ext (Eq. 17, and the paper's 330 mV at 0.91 mA
 *     with R_ext = 360 ohm); Eq. 21 as printed, I (R_int + R_ext), is returned beside it;
 *   - M_ox is kept in [0, M_total (1 - 1e-12)] after each step, so that M_red stays positive.
 * F = 96485.33212 C/mol and R = 8.314462618 J/(mol K) (exact in the 2019 SI).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    double M_total, Y, gamma, m, q_max, K_Mox, I_0, E_0, R_ext, R_int, eps, A_a, T, V_a, dt;
    int substeps;
} orc_electro;

/* out: M_ox, M_red, q_a, n_conc, n_act, I_cell, V (I R_ext), V_eq21 (I (R_int + R_ext)) */
ORC_API void orc_electro_update(const orc_electro *e, double S, double C_bio, double M_ox,
                                double *out)
{
    const double F = 96485.33212, R = 8.314462618;
    double q_a = 0.0, n_conc = 0.0, n_act = 0.0, I = 0.0;
    for (int step = 0; step < e->substeps; ++step) {
        /* Eq. 14 */
        double M_red = e->M_total - M_ox;
        /* Eq. 16 (double Monod) */
        q_a = e->q_max * S * (M_ox / (M_ox + e->K_Mox));
        /* Eq. 18 (Nernst) */
        n_conc = (R * e->T / F) * log(e->M_total / M_red);
        /* Eq. 20 with Eq. 19 inside: bisection on g(I), which is increasing in I */
        double lo = -10.0 * fabs(e->E_0) / (e->R_int + e->R_ext) - 1.0;
        double hi = -lo;
        for (int it = 0; it < 400; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break; /* no double left between the bounds */
            double act = mid / (e->A_a * e->I_0) * (R * e->T / (e->m * F)) * (M_ox / M_red);
            double rhs = (e->E_0 - n_conc - act) / (e->R_int + e->R_ext) * (M_red / (e->eps + M_red));
            if (mid - rhs > 0.0) hi = mid; else lo = mid;
        }
        I = 0.5 * (lo + hi);
        /* Eq. 19 at the root */
        n_act = I / (e->A_a * e->I_0) * (R * e->T / (e->m * F)) * (M_ox / M_red);
        /* Eq. 15 */
        M_ox = M_ox - e->dt * e->Y * q_a / 86400.0 +
               e->dt * e->gamma * I / (e->m * F) / (e->V_a * C_bio);
        if (M_ox < 0.0) M_ox = 0.0;
        if (M_ox > e->M_total * (1.0 - 1e-12)) M_ox = e->M_total * (1.0 - 1e-12);
    }
    out[0] = M_ox;
    out[1] = e->M_total - M_ox;
    out[2] = q_a;
    out[3] = n_conc;
    out[4] = n_act;
    out[5] = I;
    out[6] = I * e->R_ext;
    out[7] = I * (e->R_int + e->R_ext);
}

ORC_API int orc_electro_size(void) { return (int)sizeof(orc_electro); }

ORC_API int orc_params_size(void) { return (int)sizeof(orc_params); }
ORC_API int orc_result_size(void) { return (int)sizeof(orc_result); }
