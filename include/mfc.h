/*
 * mfc.h — C ABI of the GB300 (sm_103a) library for the coupled flow + substrate-transport
 * lattice Boltzmann solvers of the microbial fuel cell model of Tsompanas et al.,
 * "Modelling Microbial Fuel Cells using lattice Boltzmann methods" (arXiv 1802.07525).
 *
 * What the library computes (Sec. 3 of the paper, steps 2 and 3 of the model loop):
 *   - flow: BGK lattice Boltzmann (Eq. 4) with the equilibrium of Eq. 5, moments Eqs. 9-10 and
 *     half-way bounce-back on walls, electrode and biofilm (Eq. 11); D2Q9 in 2-D, D3Q19 in 3-D;
 *   - transport: BGK advection-diffusion lattice Boltzmann (Eq. 12, concentration Eq. 13) of
 *     the substrate, driven by the flow velocity, zero flux on solids, Dirichlet inlet;
 *     D2Q5 / D3Q7; a first-order consumption k*C on biofilm (sink) nodes;
 *   - the consumption summed over the lattice (the current of the anode in lattice units,
 *     the chain of Eqs. 16 and 20), and the residuals that decide steady state.
 *
 * Conventions shared by every call:
 *   - Lattice units: dx = dt = 1, reference density 1.  The flow axis is x in 2-D and z in 3-D;
 *     the inlet is at its low end.
 *   - Node order: x fastest, then y, then z; N = nx*ny*nz.  Host arrays are dense in this order.
 *   - Node classes (uint8 per node): bit 0 (1) blocked for the flow, bit 1 (2) blocked for
 *     transport, bit 2 (4) consumption node.  Electrode = 3, biofilm next to electrode = 4
 *     (consumes, open to flow) or 5 (consumes, impermeable to flow).
 *   - Boundary kinds per axis: MFC_BC_WALL (half-way bounce-back walls outside the first and
 *     last layer), MFC_BC_PERIODIC, MFC_BC_INOUT (flow axis only: moving-wall bounce-back
 *     inlet at u_in; outlet at density rho_out with the velocity of the last layer; transport
 *     inlet at c_in, zero-gradient or Dirichlet-c_out outlet).
 *   - Ownership: the library allocates and owns all device memory of a lattice; every host
 *     pointer belongs to the caller and is only read or written during the call.
 *   - Streams: a lattice runs on the stream given in its descriptor (NULL: a stream the
 *     library creates).  Stepping calls are asynchronous on that stream; read calls and
 *     mfc_solve_steady block until their results are on the host.
 *   - Errors: every call returns an mfc_status; nothing aborts or exits.  A CUDA error is
 *     recorded on the lattice and returned by that call and every later call on it.
 *   - Precision: flow populations are stored as deviations from rest (f_i - w_i), transport
 *     populations as they are (g_i), in FP32 (MFC_FP32) or FP16 (MFC_FP16_DEV) with FP32
 *     arithmetic and FP32 fields, or in FP64 with FP64 arithmetic and FP64 fields (MFC_FP64:
 *     the same kernels instantiated in double, a parity reference for the FP64 method of the
 *     paper, single lattices only); residual, mass and current sums are FP64.
 */
#ifndef MFC_H
#define MFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MFC_API __attribute__((visibility("default")))
#else
#define MFC_API
#endif

typedef struct mfc_lattice mfc_lattice; /* opaque; owns its device memory */

typedef enum {
    MFC_OK = 0,
    MFC_ERR_ARG = 1,          /* invalid argument (size, pointer, parameter range) */
    MFC_ERR_OOM = 2,          /* device allocation failed */
    MFC_ERR_OOM_BUDGET = 3,   /* the request does not fit the memory budget of a batch */
    MFC_ERR_CUDA = 4,         /* a CUDA call failed; see mfc_last_error */
    MFC_NOT_CONVERGED = 5,    /* step cap reached before the residuals fell below tolerance */
    MFC_ERR_NONFINITE = 6,    /* a residual, mass or current sum was not finite */
    MFC_ERR_TIMEOUT = 7,      /* the host-side wall-clock limit of a solve was reached */
    MFC_ERR_STATE = 8,        /* call not valid in the object's current state */
    MFC_PENDING = 9,          /* a batch request has not finished yet */
    MFC_ERR_UNSTABLE = 10     /* at a check, a flow-open node moved at or above the lattice sound
                                 speed (|u|^2 >= 1/3) or had rho <= 0: the flow has left the range
                                 of the low-Mach BGK equilibrium (Eq. 5) and the solve stops there,
                                 before it turns non-finite */
} mfc_status;

enum { MFC_BC_WALL = 0, MFC_BC_PERIODIC = 1, MFC_BC_INOUT = 2 };
enum { MFC_FP32 = 0, MFC_FP16_DEV = 1, MFC_FP64 = 2 };
enum { MFC_SEQUENTIAL = 0, MFC_CONCURRENT = 1 };
enum { MFC_OUTLET_ZERO_GRADIENT = 0, MFC_OUTLET_DIRICHLET = 1 };
enum { MFC_POP_FLOW = 0, MFC_POP_ADE = 1, MFC_FIELD_VELOCITY = 2 };

typedef struct {
    int dim;          /* 2 or 3 */
    int nx, ny, nz;   /* lattice size; nz = 1 in 2-D */
    int bc[3];        /* boundary kind per axis */
    int precision;    /* MFC_FP32, MFC_FP16_DEV or MFC_FP64 (population storage; MFC_FP64
                         also computes in FP64); batches take MFC_FP32 or MFC_FP16_DEV */
    int ade_q;        /* transport velocity set: 0 for the default (D2Q5 in 2-D, D3Q7 in 3-D,
                         with the linear equilibrium), or 9 in 2-D: D2Q9 with the equilibrium
                         of Eq. 5, C in place of rho (the text after Eq. 12); batches take the
                         default only */
    int cut[2];       /* slab decomposition along the flow axis: cut[0] (cut[1]) = 1 makes the
                         low (high) face of the flow axis a cut to a neighbouring slab, whose
                         crossing populations arrive through mfc_halo_unpack instead of the
                         axis' boundary kind (0 for a whole lattice; a lattice with a cut may not
                         be periodic along the flow axis; batches take no cuts) */
    void *stream;     /* cudaStream_t, or NULL for a library-owned stream */
} mfc_lattice_desc;

typedef struct {
    double tau;        /* flow relaxation time (Eq. 4), > 0.5; viscosity (tau - 1/2)/3 */
    double tau_c;      /* transport relaxation time tau_D (Eq. 12), > 0.5 */
    double u_in;       /* inlet speed along the flow axis */
    double rho_in;     /* density of the moving wall forming the inlet (normally 1) */
    double rho_out;    /* outlet density (pressure reference, normally 1) */
    double c_in;       /* inlet substrate concentration */
    double c_out;      /* outlet concentration for a Dirichlet outlet */
    double k_sink;     /* consumption rate on sink nodes per unit concentration, in [0, 1): the
                          first-order rate k_sink*C, or the low-concentration slope of the
                          saturating rate below */
    double u_scale;    /* factor on the flow velocity seen by transport (1 = same units) */
    int ade_outlet;    /* MFC_OUTLET_ZERO_GRADIENT or MFC_OUTLET_DIRICHLET */
    double k_half;     /* half-saturation concentration K_s of the substrate factor of Eq. 16
                          (>= 0, lattice concentration units): the consumption on a sink node is
                          k_sink*C*K_s/(K_s + C), i.e. q_max*C/(C + K_s) with q_max = k_sink*K_s
                          and the mediator factor folded into k_sink; 0 = first order */
} mfc_params;

/* Residual of a check at step n: the mean relative change per step since the previous check m,
 *     r = ||v^n - v^m||_2 / ((n - m) ||v^n||_2)   (sums over the open nodes, in FP64),
 * for v = u (flow) and v = C (transport).  m is the previous check of the same solve, or, for
 * the first check, the last step run before the call (every stepping call stores its last
 * step's fields).  With K = 1 this is the per-step change; a longer interval averages out the
 * step-to-step rounding jitter of FP32 / FP16 populations near steady state. */
typedef struct {
    double tol_flow;   /* flow steady when its residual r < tol_flow */
    double tol_ade;    /* transport steady when its residual r < tol_ade */
    long max_steps;    /* step cap per solver (sequential) or for both (concurrent) */
    int check_every;   /* K >= 1: a check every K steps and at the step cap */
    int mode;          /* MFC_SEQUENTIAL (flow to steady, then transport) or MFC_CONCURRENT */
    double timeout_s;  /* host wall-clock limit; <= 0 for none */
} mfc_solve_opts;

typedef struct {
    long steps_flow, steps_ade; /* steps taken by each solver in this call */
    double res_flow, res_ade;   /* residuals at the last check */
    double current;             /* sum over consumption nodes of the consumption (k*C, or
                                   k*C*K_s/(K_s + C)) at the last check */
    double mass;                /* sum of rho over flow-open nodes at the last check */
    double substrate;           /* sum of C over transport-open nodes at the last check */
    int status;                 /* the mfc_status the call returned */
} mfc_solve_result;

/* ---- lattice life cycle ---------------------------------------------------------------- */

/* Allocate a lattice (populations A/B, classes, link masks, fields, reduction scratch) on the
 * current CUDA device.  Fails with MFC_ERR_ARG for bad sizes/kinds, tau or tau_c <= 0.5,
 * an INOUT kind on a cross axis; MFC_ERR_OOM when device memory is short.  The lattice
 * starts with every node open and the rest state (flow at rest, no substrate). */
MFC_API mfc_status mfc_create_lattice(const mfc_lattice_desc *desc, const mfc_params *params,
                                      mfc_lattice **out);
MFC_API mfc_status mfc_destroy_lattice(mfc_lattice *lat);

/* Replace the physical parameters (relaxation times, inlet, consumption rate, ...). */
MFC_API mfc_status mfc_set_params(mfc_lattice *lat, const mfc_params *params);

/* Copy N node classes from host memory and rebuild the link masks (Eq. 11 decides which
 * links bounce back).  reset_fields != 0: every open node returns to the rest state.
 * reset_fields == 0: populations are kept (warm start); nodes that open up start at rest,
 * nodes that become blocked drop their populations.  Class values above 7 are rejected. */
MFC_API mfc_status mfc_set_geometry(mfc_lattice *lat, const uint8_t *node_class,
                                    int reset_fields);

/* ---- stepping (asynchronous on the lattice stream) ------------------------------------- */

/* nsteps flow steps (Eq. 4).  The last one stores rho and u in the field buffers. */
MFC_API mfc_status mfc_step_flow(mfc_lattice *lat, int nsteps);
/* nsteps transport steps (Eq. 12) with the stored velocity held fixed (the paper's order).
 * The last one stores C. */
MFC_API mfc_status mfc_step_ade(mfc_lattice *lat, int nsteps);
/* nsteps fused steps of both lattices; transport uses the same step's flow velocity. */
MFC_API mfc_status mfc_step_coupled(mfc_lattice *lat, int nsteps);
/* As mfc_step_coupled, but the stored fields stay those of the last call that stored them (a
 * check, or a stepping call's last step): for callers that check on their own schedule one step
 * at a time, such as the slabs of a decomposed lattice between their checks. */
MFC_API mfc_status mfc_step_coupled_plain(mfc_lattice *lat, int nsteps);

/* Iterate to steady state (Sec. 4: "enough time steps until an equilibrium is reached"),
 * checking the residuals every K steps with CUDA-graph replays of K steps.  Blocks.
 * Returns MFC_OK, MFC_NOT_CONVERGED, MFC_ERR_NONFINITE, MFC_ERR_UNSTABLE (first check with a
 * node at or above the sound speed or at rho <= 0) or MFC_ERR_TIMEOUT; out (optional) is
 * filled in every case. */
MFC_API mfc_status mfc_solve_steady(mfc_lattice *lat, const mfc_solve_opts *opts,
                                    mfc_solve_result *out);

/* ---- biofilm growth between steady solves ---------------------------------------------- */

/* Grow biofilm: every open node (class 0) with a consumption node among its flow-lattice
 * neighbours, local concentration C > c_thresh and a draw below prob becomes impermeable
 * biofilm (class 5).  Draw: splitmix64(seed ^ (cycle << 32) ^ node), converted when its top
 * 53 bits are below prob * 2^53.  Decisions read the classes from before the pass and the
 * concentration field of the last stepping call.  The link masks are rebuilt (warm start).
 * n_converted (optional, host) receives the count; it blocks for that copy.  This is a
 * simplified stand-in for the agent-based biofilm model of Sec. 3.3. */
MFC_API mfc_status mfc_biofilm_grow(mfc_lattice *lat, uint64_t seed, uint64_t cycle,
                                    double prob, double c_thresh, long *n_converted);

/* ---- agent-based biofilm (Sec. 3.3) ------------------------------------------------------ */

/* Biofilm formation between steady solves, on a biomass concentration C^bio per node (mg
 * biomass / L) that the lattice keeps in device memory.  One call runs, in this order:
 *   attachment: the k_ata front nodes with the smallest keys get C^bio = C_0^bio.  The front is
 *     the open nodes (class 0) without biomass that have an electrode node (class bits 0 and 1)
 *     among their flow-lattice neighbours; the key of node k is (top 32 bits of h) << 32 | k,
 *     h = splitmix64(splitmix64(seed ^ 0x6174746163680000) ^ (cycle << 32) ^ k), so the choice is
 *     exact and repeatable; every front node when there are fewer than k_ata;
 *   growth (the double Monod law of Eq. 16): every transport-open node with biomass,
 *     C^bio <- C^bio (1 + growth * s), s = C+ / (C+ + k_half), C+ = max(C, 0), C the substrate
 *     concentration of the last stepping call;
 *   spreading: the nodes above c_max_bio when spreading starts, in increasing node order; one
 *     still above it when reached passes fr_spr of its biomass to a free neighbour (an open node
 *     without biomass) drawn at random, or, with none free, to the first cell of a loop-erased
 *     random walk through the biofilm (steps onto the electrode or out of the lattice are lost)
 *     that ends on a free cell, after every cell with biomass on the walk's path has passed its
 *     biomass one cell on towards that free cell; a walk of max_walk steps gives up.  Draw n of
 *     the pass is splitmix64(splitmix64(seed ^ 0x7370726561640000 ^ (cycle << 32)) ^ n), a choice
 *     among m options taking (draw >> 32) % m;
 *   classes: every non-electrode node with biomass becomes biofilm, impermeable to the flow and
 *     consuming substrate (class 5); the link masks are rebuilt (warm start).
 * Attachment, growth and the class update are data-parallel kernels; spreading, whose events
 * move biomass along chains one after another, runs as one device thread.  Growth and the
 * spreading split are FP64 without contraction; every decision is integer.  Blocks until done. */
typedef struct {
    uint64_t seed;
    int k_ata;          /* front nodes attached per call (Table 1: 200), >= 0 */
    double c0_bio;      /* C_0^bio, the biomass of an attached node (Table 1: 450), > 0 */
    double c_max_bio;   /* C_max^bio, the spreading threshold (Table 1: 512.5), > 0 */
    double fr_spr;      /* fraction of a spreading node's biomass moved (Table 1: 0.4), [0, 1] */
    double growth;      /* relative growth per call at saturating substrate: the double Monod
                           rate of Eq. 16 with its mediator factor, times a biomass yield and the
                           call's time span (not given by the paper), >= 0 */
    double k_half;      /* K_s of Eq. 16 in lattice concentration units, > 0 */
    int max_walk;       /* steps a spreading walk may take, 1..65536 */
} mfc_agent_params;

typedef struct {
    long long attached;       /* nodes attached by this call */
    long long front;          /* front nodes it chose among */
    long long spread;         /* spreading events */
    long long walks_failed;   /* walks that gave up */
    long long walk_steps;     /* walk steps taken */
    long long biofilm_nodes;  /* nodes with biomass after the call */
    double total_biomass;     /* sum of C^bio after the call (FP64) */
} mfc_agent_stats;

/* One biofilm-formation step (above).  Fails with MFC_ERR_ARG for a parameter out of range or a
 * lattice of 2^31 nodes or more.  out is optional.  The biomass starts at zero everywhere. */
MFC_API mfc_status mfc_agent_step(mfc_lattice *lat, const mfc_agent_params *p, uint64_t cycle,
                                  mfc_agent_stats *out);
/* C^bio of every node, N doubles in host memory (zeros before the first step or write). */
MFC_API mfc_status mfc_read_biomass(mfc_lattice *lat, double *host);
/* Replace C^bio by N host doubles (each finite and >= 0).  The classes follow at the next
 * mfc_agent_step; biomass on electrode nodes is never grown or spread and makes no biofilm
 * (the statistics still count it). */
MFC_API mfc_status mfc_write_biomass(mfc_lattice *lat, const double *host);

/* ---- bio-electrochemical model of the anode (host only) -------------------------------- */

/* The electrical side of the model (Sec. 3.2, Eqs. 14-21), lumped over the anode and advanced
 * once per model iteration (one hour of real time, Sec. 4) from what the steady lattice solve
 * gives: the mean substrate factor C/(C + K_s) over the biofilm (for a lattice solved with the
 * saturating consumption, current / (k_sink * k_half * consumption nodes)).  Units: mediator
 * amounts per unit biomass (mg mediator / mg biomass), q_max per day, currents in A, voltages
 * in V, resistances in ohm, V_a in L, C^bio in mg biomass / L, time steps in s.  Host arithmetic
 * in double; no device work, no allocation. */
typedef struct {
    double m_total;     /* M_total: total intracellular mediator (Table 1: 0.05) */
    double mediator_yield; /* Y: mediator yield, mg mediator / mg substrate (0.5687) */
    double gamma;       /* mediator molar mass, mg / mol (663400) */
    double m_electrons; /* m: electrons per reduced mediator (2) */
    double q_max;       /* maximum consumption rate, mg substrate / (mg biomass day) (8.48) */
    double k_mox;       /* K_Mox: half saturation of the oxidised mediator (0.02 M_total) */
    double i0;          /* I_0: exchange current density, A / m^2 (0.001) */
    double e0;          /* E_0: open-circuit voltage, V (0.7) */
    double r_ext;       /* external (load) resistance, ohm (360) */
    double r_int;       /* internal resistance, ohm (360) */
    double epsilon;     /* epsilon of Eq. 20, same units as M_red (not given by the paper) */
    double area;        /* A_a: anode surface area, m^2 (not given by the paper) */
    double temperature; /* T, K (not given by the paper) */
    double volume;      /* V_a: anode compartment volume, L (17 x 60 x 65 mm = 0.0663 L) */
    double dt;          /* time step of Eq. 15, s */
    int substeps;       /* Eq. 15 steps per call (each of dt seconds), >= 1 */
} mfc_electro_params;

typedef struct {
    double m_ox;      /* M_ox after the call (Eq. 15) */
    double m_red;     /* M_red = M_total - M_ox after the call (Eq. 14) */
    double q_a;       /* consumption rate of the last step, mg substrate / (mg biomass day) (Eq. 16) */
    double n_conc;    /* concentration overpotential of the last step, V (Eq. 18) */
    double n_act;     /* activation overpotential of the last step, V (Eq. 19) */
    double i_cell;    /* current of the last step, A (Eq. 20 solved for I, Eqs. 17-19 inside) */
    double v_cell;    /* I_cell * R_ext, V: the voltage across the load (Eq. 17, and the paper's
                         reported 330 mV at 0.91 mA) */
    double v_eq21;    /* I_cell * (R_int + R_ext), V: Eq. 21 as printed */
} mfc_electro_result;

/* Table 1's values, and for the constants the paper does not give: epsilon = 0.01 (mg mediator /
 * mg biomass), A_a = 0.0031 m^2 (the electrode's 48 x 65 mm face), T = 298.15 K; V_a = 0.0663 L;
 * one model iteration (an hour) as 3600 steps of dt = 1 s (an explicit step of an hour would
 * overshoot the mediator balance, whose relaxation time is about 20 s at these values).
 * Returns MFC_ERR_ARG for a NULL pointer. */
MFC_API mfc_status mfc_electro_default_params(mfc_electro_params *p);

/* Advance the mediator balance by p->substeps steps of p->dt seconds, each in the paper's order:
 *   M_red = M_total - M_ox                                                          (Eq. 14)
 *   q_a = q_max * S * M_ox / (M_ox + K_Mox), S = substrate_factor                    (Eq. 16)
 *   n_conc = (R T / F) ln(M_total / M_red)                                          (Eq. 18)
 *   I = (E_0 - n_conc - n_act) / (R_int + R_ext) * M_red / (epsilon + M_red)        (Eq. 20)
 *     with n_act = I / (A_a I_0) * R T / (m F) * M_ox / M_red (Eq. 19), which is linear in I,
 *     so I = (E_0 - n_conc) s / (R_int + R_ext + a s), s = M_red / (epsilon + M_red),
 *     a = R T / (m F A_a I_0) * M_ox / M_red
 *   M_ox += dt * (-Y q_a / 86400 + gamma I / (m F V_a C^bio))                         (Eq. 15)
 * M_ox stays in [0, M_total] (an explicit step that would leave it is cut at the bound).
 * substrate_factor in [0, 1]; c_bio > 0 (mg biomass / L); m_ox in [0, M_total).  out receives
 * the state after the call and the last step's rates.  Returns MFC_ERR_ARG for a NULL pointer or
 * an argument out of range. */
MFC_API mfc_status mfc_electro_update(const mfc_electro_params *p, double substrate_factor,
                                      double c_bio, double m_ox, mfc_electro_result *out);

/* ---- reading results and checkpointing (blocking) --------------------------------------- */

/* Fields of the last stepping call, as doubles in host memory (each pointer may be NULL):
 * rho[N] (flow moment Eq. 9, 0 on flow-blocked nodes), u[dim*N] (component-major, Eq. 10,
 * 0 on flow-blocked nodes), c[N] (Eq. 13, 0 on transport-blocked nodes), current[1] (sum of
 * k*C over consumption nodes at the last residual check or solve). */
MFC_API mfc_status mfc_read_fields(mfc_lattice *lat, double *rho, double *u, double *c,
                                   double *current);

/* Raw populations for checkpoint/resume and parity checks, as absolute values in doubles:
 * which = MFC_POP_FLOW (Q_flow*N, direction-major), MFC_POP_ADE (Q_ade*N), or
 * MFC_FIELD_VELOCITY (dim*N, the velocity that transport steps read).  Blocked nodes read 0. */
MFC_API mfc_status mfc_read_populations(mfc_lattice *lat, int which, double *host);
MFC_API mfc_status mfc_write_populations(mfc_lattice *lat, int which, const double *host);

/* Wait for all work queued on the lattice stream. */
MFC_API mfc_status mfc_synchronize(mfc_lattice *lat);

/* ---- launch variants ---------------------------------------------------------------------- */

/* How the step kernel is launched: `block` (128 or 256) threads along a row per block, one node
 * per thread (with FP16 storage and 32-bit offsets, plain coupled steps take two rows per thread,
 * nodes (x, y) and (x, y + 1), with paired FP32 arithmetic).  Every choice computes the same
 * arithmetic; the paired form groups the FP32 operations differently, so it agrees to FP32
 * rounding. */
typedef struct {
    int block;
    int offsets32;  /* 1 (default): the plain step forms its element offsets in 32 bits where every
                       population array has fewer than 2^31 elements (one multiply-add per address);
                       0: 64-bit offsets always, one node per thread */
} mfc_launch;

/* Select the launch shape (waits for queued work; captured step graphs are rebuilt). */
MFC_API mfc_status mfc_set_launch(mfc_lattice *lat, const mfc_launch *launch);
MFC_API mfc_status mfc_get_launch(mfc_lattice *lat, mfc_launch *launch);

/* ---- slab decomposition (one lattice split along the flow axis) ------------------------- */

/* A lattice too large for one GPU splits along the flow axis into slabs, one per GPU, each a
 * lattice whose faces towards its neighbours are cuts (mfc_lattice_desc.cut).  After every step,
 * each slab packs the populations that leave it through a cut face and the neighbour unpacks them
 * into its ghost layer, where its next step pulls them; the check sums of a step are summed over
 * the slabs (FP64) before the residual test.  Side 0 is the low face of the flow axis, side 1 the
 * high face.  The population values cross in their storage type (FP32, FP16 or FP64), so a slab
 * run computes exactly what the whole lattice computes.  Buffers are device memory of the caller,
 * used in stream order on the lattice stream. */

/* Bytes of the halo of one side: (crossing flow planes + crossing transport planes) x the nodes of
 * a cross-section x the storage size. */
MFC_API mfc_status mfc_halo_bytes(mfc_lattice *lat, int side, size_t *bytes);
/* Queue the copy of the populations leaving through face `side` (the current state of the layer
 * next to it) into dev_buf, direction-major then cross-section in node order. */
MFC_API mfc_status mfc_halo_pack(mfc_lattice *lat, int side, void *dev_buf);
/* Queue the copy of a neighbour's packed populations (its opposite side) into the ghost layer
 * beyond face `side`, with the periodic images of the cross axes. */
MFC_API mfc_status mfc_halo_unpack(mfc_lattice *lat, int side, const void *dev_buf);
/* Node classes of the neighbour's layer next to face `side` (host, one cross-section: ny bytes in
 * 2-D, nx*ny in 3-D): they decide which links across the cut bounce back (Eq. 11).  Rebuilds the
 * link masks (warm start).  Before the first call a cut sees open nodes.  Blocks. */
MFC_API mfc_status mfc_set_halo_classes(mfc_lattice *lat, int side, const uint8_t *plane);
/* nsteps fused steps, the last one a check step; sums[9] (host) receives that step's FP64 sums
 * over this lattice: sum |u - u_prev|^2, sum |u|^2, sum rho, sum (C - C_prev)^2, sum C^2, sum C,
 * the consumption, the count of non-finite values and the count of nodes outside the range of
 * the scheme (u_prev, C_prev: the fields of the previous check or stepping call).  Blocks. */
MFC_API mfc_status mfc_step_check_sums(mfc_lattice *lat, int nsteps, double *sums);

/* ---- checking builds ---------------------------------------------------------------------- */

/* The library can be built with MFC_CHECK_BOUNDS (paper_1802_07525_gb300.build with
 * check_bounds=True: _lib/libmfc_check.so), a debugging build standing in for a memory checker:
 * the step kernels test every element offset against the array they address and record the first
 * one out of range (the access goes to an unused element instead), which the next synchronising
 * call on the lattice returns as MFC_ERR_CUDA with the kernel line and the offset; and every
 * device buffer of a lattice sits between two 256-byte guard regions of a fixed pattern.
 * mfc_check_build returns 1 in such a build, 0 otherwise. */
MFC_API int mfc_check_build(void);
/* Checking builds: *bad receives the number of guard bytes of the lattice's buffers that no longer
 * hold their pattern (a write past the end or before the start of a buffer).  Other builds: 0.
 * Blocks. */
MFC_API mfc_status mfc_check_canaries(mfc_lattice *lat, long long *bad);

/* ---- sums without allocation ------------------------------------------------------------ */

/* For callers that cannot allocate device memory (code inside another framework's memory pool
 * or under a fixed device-memory budget, where a raw cudaMalloc would break the accounting or is
 * not allowed, and paths that must not risk an allocation failure).  The paper has no
 * counterpart: this is the check-step reduction of mfc_solve_steady (the eight FP64 sums and
 * the two residuals) applied to fields the caller already holds in device memory.
 *
 * Inputs (device pointers, dense, x fastest): node_class[n] (bit 0 flow-blocked, bit 1
 * transport-blocked, bit 2 consumption), rho[n], u[dim*n] and u_prev[dim*n] (component-major),
 * c[n] and c_prev[n].  Output: out[10] in device memory, the sums sum |u-u_prev|^2, sum |u|^2,
 * sum rho (flow-open nodes), sum (c-c_prev)^2, sum c^2, sum c (transport-open nodes), sum over
 * consumption nodes of k_sink*c (the first-order law only: for a lattice with k_half > 0 this is
 * not the current mfc_solve_steady reports), the count of non-finite values, then the flow and
 * transport relative changes ||u - u_prev|| / ||u|| and ||c - c_prev|| / ||c|| between the two
 * snapshots.  These are not divided by the number of steps between the snapshots: divide them
 * by it to compare with the per-step residuals of mfc_solve_steady.  Queued on `stream`
 * (cudaStream_t; NULL for the legacy default stream).  A launch failure of this call returns
 * MFC_ERR_CUDA; an error pending from the caller's earlier work is neither returned nor cleared.
 *
 * It allocates nothing: its per-block partial sums live in a file-scope device array of 512 KiB
 * (256 nodes per block, 8192 blocks) that every GPU which loads the library holds until the
 * process exits, so n is limited to 2,097,152 nodes (MFC_ERR_ARG above that, or for dim not 2/3
 * or a NULL pointer).  The first call on a device looks up the array's device address (one
 * cudaGetSymbolAddress); make that first call before any stream capture.  Every call on a GPU
 * shares that GPU's array and it keeps the last call's partials: two calls whose kernels can
 * run at the same time on one GPU (for instance on different streams) race on it, so order them
 * (same stream, or an event between them).  Each call writes every partial it reads, so nothing
 * needs clearing between calls. */
MFC_API mfc_status mfc_field_sums_noalloc(long long n, int dim, const uint8_t *node_class,
                                          const double *rho, const double *u, const double *u_prev,
                                          const double *c, const double *c_prev, double k_sink,
                                          double *out, void *stream);

/* ---- batches: many steady solves sharing the GPU (continuous batching) ------------------ */

/* A batch runs steady solves (mfc_solve_steady with MFC_CONCURRENT) of many lattices at once.
 * Requests are admitted first come, first served, as instance slots and device memory free up
 * (each request's device memory, mfc_lattice_bytes plus the read-back staging when fields are
 * asked for, counts against budget_bytes); admitted instances stay resident on the device and
 * advance together, every lattice of every instance in one launch per step and dimension (a
 * fixed grid of a few blocks per SM walking a tile table of all instances' rows), in CUDA-graph
 * replays of K steps that end with every instance's residual check.  A finished instance
 * (converged, at its step cap, timed out, non-finite or out of range) leaves at the end of its
 * block; its fields are copied to the caller's buffers while the next block runs, and its memory
 * goes back to the batch's pool after that block.  Requests that arrive while a block runs are
 * set up (lattice, classes, link masks) on a second stream during that block and join the next
 * one, so the host work between blocks overlaps the GPU.
 *
 * What a request gets does not depend on what else runs: every instance steps and checks
 * exactly as it would alone in a batch with the same K and block, bit for bit.  Against
 * mfc_solve_steady with check_every = K, the checks fall on the same steps; the step cap is
 * taken in whole blocks (a batch solve ends at the first check at or after max_steps).
 *
 * Threads: submit, poll, wait and stats may be called from any thread.  The engine runs either
 * on the caller's thread (mfc_batch_run, until nothing is queued or running) or on a library
 * thread (mfc_batch_start ... mfc_batch_stop).  All device work runs on the batch's stream. */
typedef struct mfc_batch mfc_batch; /* opaque */

typedef struct {
    size_t budget_bytes;  /* device memory for instances; 0 = 90% of the free memory at create */
    int precision;        /* MFC_FP32 or MFC_FP16_DEV, for every instance (MFC_FP64: MFC_ERR_ARG) */
    int check_every;      /* K (even, >= 2; odd values are rounded up); 0 = chosen by the autotuner */
    int block;            /* threads per tile: 64, 128 or 256; 0 = chosen by the autotuner */
    int max_instances;    /* instance slots, 1..4096; 0 = 256 */
    void *stream;         /* cudaStream_t, or NULL for a library-owned stream */
} mfc_batch_opts;

typedef struct {
    mfc_solve_result result; /* as mfc_solve_steady fills it (steps in whole blocks) */
    double t_submit;         /* mfc_clock() at submission */
    double t_admit;          /* when the instance was created on the device */
    double t_done;           /* when the result and fields were ready */
} mfc_batch_result;

typedef struct {
    long long submitted, completed, running, queued;
    long long blocks;           /* graph replays run */
    long long instance_steps;   /* sum over instances of the steps they took */
    size_t bytes_in_use, bytes_peak, budget_bytes;
    int check_every, block, grid; /* the launch the batch runs (after autotuning) */
} mfc_batch_stats;

MFC_API mfc_status mfc_batch_create(const mfc_batch_opts *opts, mfc_batch **out);
/* Stops the engine thread, abandons unfinished requests and frees every instance. */
MFC_API mfc_status mfc_batch_destroy(mfc_batch *batch);
/* Queue a steady solve.  desc: the lattice (its precision must be the batch's; its stream is
 * ignored); params as for mfc_create_lattice; node_class: N classes, copied during the call;
 * opts: tolerances, max_steps and timeout_s (from admission) as for mfc_solve_steady, mode must
 * be MFC_CONCURRENT, check_every is ignored (the batch's K applies).  rho, u, c: optional host
 * buffers (N, dim*N, N doubles, as mfc_read_fields fills them) that the batch fills when the
 * solve ends; they must stay valid until then.  *ticket identifies the request.  Fails with
 * MFC_ERR_ARG for a bad request (including a lattice whose largest population array, the larger
 * set's Q times the pitched plane, reaches 2^31 elements: the batch kernel's offsets are 32-bit)
 * and MFC_ERR_OOM_BUDGET when it can never fit the budget. */
MFC_API mfc_status mfc_batch_submit(mfc_batch *batch, const mfc_lattice_desc *desc,
                                    const mfc_params *params, const uint8_t *node_class,
                                    const mfc_solve_opts *opts, double *rho, double *u, double *c,
                                    long long *ticket);
/* MFC_PENDING while the request runs or waits; otherwise the solve's status (as
 * mfc_solve_steady returns it) with *out filled, and the ticket is released. */
MFC_API mfc_status mfc_batch_poll(mfc_batch *batch, long long ticket, mfc_batch_result *out);
/* As poll, waiting up to timeout_s seconds (< 0: no limit) for the request to finish. */
MFC_API mfc_status mfc_batch_wait(mfc_batch *batch, long long ticket, double timeout_s,
                                  mfc_batch_result *out);
/* Run the engine on the calling thread until no request is queued or running. */
MFC_API mfc_status mfc_batch_run(mfc_batch *batch);
/* Run the engine on a library thread, which admits requests as they arrive. */
MFC_API mfc_status mfc_batch_start(mfc_batch *batch);
/* Stop the engine thread at the end of its current turn (requests stay queued or resident; a
 * block it queued may still be in flight, and the next mfc_batch_run or mfc_batch_start takes its
 * results). */
MFC_API mfc_status mfc_batch_stop(mfc_batch *batch);
MFC_API mfc_status mfc_batch_get_stats(mfc_batch *batch, mfc_batch_stats *out);
/* Text of the batch's last error. */
MFC_API const char *mfc_batch_last_error(mfc_batch *batch);
/* Seconds on the library's monotonic clock (the clock of the batch time stamps). */
MFC_API double mfc_clock(void);

/* ---- introspection --------------------------------------------------------------------- */

/* Number of nodes open for flow and for transport (computed at mfc_set_geometry). */
MFC_API mfc_status mfc_active_nodes(mfc_lattice *lat, long *flow_open, long *ade_open);
/* Bytes of device memory the lattice holds. */
MFC_API mfc_status mfc_device_bytes(mfc_lattice *lat, size_t *bytes);
/* Device memory a lattice with this descriptor would allocate (for admission control). */
MFC_API size_t mfc_lattice_bytes(const mfc_lattice_desc *desc);
MFC_API const char *mfc_status_string(mfc_status s);
/* Text of the last error recorded on the lattice (or of the last create failure when lat is
 * NULL); the pointer stays valid until the next call on that lattice. */
MFC_API const char *mfc_last_error(mfc_lattice *lat);
/* Library version, e.g. "mfc 0.1 sm_103a". */
MFC_API const char *mfc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MFC_H */
