// Fused pull-scheme stream-collide kernels of the coupled flow + substrate lattice Boltzmann
// solvers (Tsompanas et al., arXiv 1802.07525, Sec. 3.1), their residual/current reductions,
// link-mask construction, field conversion and the biofilm growth rule.
//
// One thread updates one node per row it visits.  Flow (Eq. 4 with Eq. 5, moments Eqs. 9-10):
// the populations arriving at x are gathered from x - c_i in the previous buffer (pull), with
// half-way bounce-back (Eq. 11) where the link mask says the source is a wall or blocked node,
// the moving-wall inlet and the pressure outlet at the ends of the flow axis; then BGK
// relaxation to the equilibrium.  Transport (Eq. 12, moment Eq. 13): the same gather on the
// D2Q5 / D3Q7 set with zero-flux bounce-back on transport-blocked nodes, an equilibrium inlet
// ghost at c_in and a zero-gradient (or Dirichlet) outlet, BGK relaxation to the linear
// equilibrium w_i C (1 + c_i.u / cs^2), and the consumption w_i k C on sink nodes.
//
// Flow populations are stored as deviations from rest (f_i - w_i) so that FP32 (or FP16) keeps
// the small velocity-carrying part; transport populations as g_i - w_i c_ref (c_ref = 0 in FP32,
// where the no-substrate start state is then exact).  Arithmetic is FP32.  The rest population
// of each lattice is written as the conserved total minus the moving ones.  Check steps accumulate
// the residual, mass, substrate and current sums in FP64 (warp shuffles, then shared memory,
// one partial per block; a single-block kernel adds the partials in a fixed order).
#pragma once

#include "lbm_lattice.cuh"

namespace mfc {

enum : int { MODE_PLAIN = 0, MODE_WRITE = 1, MODE_CHECK = 2 };

template <int DIM, typename ST> struct StepArgs {
    static constexpr int QF = FlowSet<DIM>::Q;
    static constexpr int QA = AdeSet<DIM>::Q;
    using LinkT = typename Links<DIM>::T;

    int nx, ny, nz;       // lattice size (nz = 1 in 2-D)
    int px;               // row pitch in elements (nx rounded up to 32)
    long long plane;      // elements per population plane = px * ny * nz
    int bc_flow_axis;     // boundary kind of the flow axis (x in 2-D, z in 3-D)
    int rows_per_block;   // consecutive (y,z) rows each block walks
    const ST *fsrc;       // flow populations, previous step, QF planes
    ST *fdst;             // flow populations, this step
    const ST *gsrc;       // transport populations, previous step, QA planes
    ST *gdst;             // transport populations, this step
    const LinkT *link;    // link mask per node
    float *fld_rho;       // rho - 1 (written on WRITE/CHECK steps)
    float *fld_u;         // DIM planes of velocity (read by frozen-velocity transport)
    float *fld_c;         // C - c_ref
    double *partials;     // NSUM doubles per block (CHECK steps)
    float omega;          // 1 / tau
    float omega_c;        // 1 / tau_c
    float k_sink;         // consumption rate
    float u_scale;        // factor on the velocity seen by transport
    float rho_out;        // outlet density
    float c_ref;          // concentration offset of the stored transport deviations
    int ade_dirichlet;    // transport outlet: 0 zero-gradient, 1 Dirichlet
    float bb_in[QF];      // moving-wall inlet term 2 w_i rho_in (c_i . u_in) / cs^2
    float gin_dev[QA];    // inlet ghost: w_i c_in (1 + c_i . u_in / cs^2) - w_i c_ref
    float gout_dev[QA];   // Dirichlet outlet ghost at c_out, same form
};

// ---- helpers ---------------------------------------------------------------------------------

template <int DIM> __device__ __forceinline__ constexpr int flow_axis() { return DIM == 2 ? 0 : 2; }

template <int DIM, typename ST>
__device__ __forceinline__ long long node_index(const StepArgs<DIM, ST> &a, int x, int y, int z)
{
    return (long long)x + (long long)a.px * ((long long)y + (long long)a.ny * z);
}

// Source of the population arriving at (x,y,z) along c_i on an edge node whose link is open.
// Returns 0: ordinary node (index in *src), 1: inlet, 2: outlet (index of the last-layer node).
template <int DIM, typename ST, typename SET>
__device__ __forceinline__ int edge_source(const StepArgs<DIM, ST> &a, int x, int y, int z, int i,
                                          long long *src)
{
    int s[3] = {x - SET::c(i, 0), y - SET::c(i, 1), z - SET::c(i, 2)};
    const int n[3] = {a.nx, a.ny, a.nz};
    constexpr int FA = flow_axis<DIM>();
    int kind = 0;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        if (s[ax] >= 0 && s[ax] < n[ax]) continue;
        if (ax == FA && a.bc_flow_axis == BC_INOUT) {
            if (s[ax] < 0) {
                kind = 1;
            } else {
                kind = 2;
                s[ax] = n[ax] - 1;
            }
        } else {  // a wall would have set the bounce-back bit, so this axis is periodic
            s[ax] = s[ax] < 0 ? s[ax] + n[ax] : s[ax] - n[ax];
        }
    }
    if (kind == 1) return 1;
    *src = node_index<DIM, ST>(a, s[0], s[1], s[2]);
    return kind;
}

// Flow outlet ghost: equilibrium deviation at rho_out with the velocity of the post-collision
// populations of last-layer node s.
template <int DIM, typename ST>
__device__ __forceinline__ float outlet_flow(const StepArgs<DIM, ST> &a, long long s, int i)
{
    using F = FlowSet<DIM>;
    float rp = 0.f, j[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < F::Q; ++m) {
        const float v = ld(a.fsrc + m * a.plane + s);
        rp += v;
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) j[ax] += F::c(m, ax) * v;
    }
    const float inv = 1.0f / (1.0f + rp);
    float cu = 0.f, uu = 0.f;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        const float u = j[ax] * inv;
        cu += F::c(i, ax) * u;
        uu += u * u;
    }
    return F::w(i) * (a.rho_out - 1.0f + a.rho_out * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
}

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum NSUM doubles over the block; thread 0 writes them to partials[block].
__device__ __forceinline__ void block_partials(double (&acc)[NSUM], double *partials)
{
    __shared__ double sh[32][NSUM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = warp_sum(acc[m]);
    if (lane == 0) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) sh[warp][m] = acc[m];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) {
            double v = lane < nwarp ? sh[lane][m] : 0.0;
            v = warp_sum(v);
            if (lane == 0) partials[(size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NSUM + m] = v;
        }
    }
}

// ---- one node ------------------------------------------------------------------------------

template <int DIM, typename ST, bool FLOW, bool ADE, int MODE, bool EDGE>
__device__ __forceinline__ void update_node(const StepArgs<DIM, ST> &a, int x, int y, int z,
                                            const long long (&off_f)[FlowSet<DIM>::Q],
                                            const long long (&off_a)[AdeSet<DIM>::Q],
                                            double (&acc)[NSUM])
{
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM>;
    using LK = Links<DIM>;
    const long long k = node_index<DIM, ST>(a, x, y, z);
    const uint32_t L = a.link[k];
    float u[3] = {0.f, 0.f, 0.f};

    if (FLOW && !(L & (1u << LK::FLOW_SELF))) {
        float d[F::Q];
        d[0] = ld(a.fsrc + k);
#pragma unroll
        for (int i = 1; i < F::Q; ++i) {
            const bool bb = (L >> i) & 1u;
            if (!EDGE) {
                const long long p = bb ? (long long)F::opp(i) * a.plane + k
                                       : (long long)i * a.plane + k - off_f[i];
                d[i] = ld(a.fsrc + p);
            } else if (bb) {
                d[i] = ld(a.fsrc + (long long)F::opp(i) * a.plane + k);
            } else {
                long long s = 0;
                const int kind = edge_source<DIM, ST, F>(a, x, y, z, i, &s);
                if (kind == 0)
                    d[i] = ld(a.fsrc + (long long)i * a.plane + s);
                else if (kind == 1)
                    d[i] = ld(a.fsrc + (long long)F::opp(i) * a.plane + k) + a.bb_in[i];
                else
                    d[i] = outlet_flow<DIM, ST>(a, s, i);
            }
        }
        float rp = 0.f, j[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < F::Q; ++i) {
            rp += d[i];
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) j[ax] += F::c(i, ax) * d[i];
        }
        const float rho = 1.0f + rp;
        const float inv = 1.0f / rho;
        float uu = 0.f;
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) {
            u[ax] = j[ax] * inv;
            uu += u[ax] * u[ax];
        }
        // BGK relaxation of the moving populations; the rest population takes what closes the
        // mass exactly (collision conserves sum_i f_i), so FP32 rounding cannot drift the mass.
        float moved = 0.f;
#pragma unroll
        for (int i = 1; i < F::Q; ++i) {
            float cu = 0.f;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) cu += F::c(i, ax) * u[ax];
            const float feq = F::w(i) * (rp + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
            const float v = kept(a.fdst, d[i] + a.omega * (feq - d[i]));
            st(a.fdst + (long long)i * a.plane + k, v);
            moved += v;
        }
        st(a.fdst + k, rp - moved);
        if (MODE != MODE_PLAIN) {
            if (MODE == MODE_CHECK) {
                double du2 = 0.0, u2 = 0.0;
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) {
                    const double un = u[ax];
                    const double dd = un - (double)a.fld_u[ax * a.plane + k];
                    du2 += dd * dd;
                    u2 += un * un;
                }
                acc[SUM_DU2] += du2;
                acc[SUM_U2] += u2;
                acc[SUM_MASS] += 1.0 + (double)rp;
                if (!isfinite(rp) || !isfinite(u2)) acc[SUM_BAD] += 1.0;
            }
            a.fld_rho[k] = rp;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) a.fld_u[ax * a.plane + k] = u[ax];
        }
    }

    if (ADE && !(L & (1u << LK::ADE_SELF))) {
        if (FLOW) {
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) u[ax] *= a.u_scale;  // 0 on flow-blocked nodes
        } else if (!(L & (1u << LK::FLOW_SELF))) {
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) u[ax] = a.fld_u[ax * a.plane + k] * a.u_scale;
        }
        float e[A::Q];
        e[0] = ld(a.gsrc + k);
#pragma unroll
        for (int i = 1; i < A::Q; ++i) {
            const bool bb = (L >> (LK::ADE_SELF + i)) & 1u;
            if (!EDGE) {
                const long long p = bb ? (long long)A::opp(i) * a.plane + k
                                       : (long long)i * a.plane + k - off_a[i];
                e[i] = ld(a.gsrc + p);
            } else if (bb) {
                e[i] = ld(a.gsrc + (long long)A::opp(i) * a.plane + k);
            } else {
                long long s = 0;
                const int kind = edge_source<DIM, ST, A>(a, x, y, z, i, &s);
                if (kind == 0)
                    e[i] = ld(a.gsrc + (long long)i * a.plane + s);
                else if (kind == 1)
                    e[i] = a.gin_dev[i];
                else
                    e[i] = a.ade_dirichlet ? a.gout_dev[i] : ld(a.gsrc + (long long)i * a.plane + s);
            }
        }
        float cp = 0.f;
#pragma unroll
        for (int i = 0; i < A::Q; ++i) cp += e[i];
        const float C = a.c_ref + cp;
        const float sink = (L & (1u << LK::SINK)) ? a.k_sink * C : 0.0f;
        // Same closure: after relaxation and consumption the populations hold C - kC exactly.
        float moved = 0.f;
#pragma unroll
        for (int i = 1; i < A::Q; ++i) {
            float cu = 0.f;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) cu += A::c(i, ax) * u[ax];
            const float geq = A::w(i) * (cp + C * cu * A::inv_cs2);
            const float v = kept(a.gdst, e[i] + a.omega_c * (geq - e[i]) - A::w(i) * sink);
            st(a.gdst + (long long)i * a.plane + k, v);
            moved += v;
        }
        st(a.gdst + k, cp - sink - moved);
        if (MODE != MODE_PLAIN) {
            if (MODE == MODE_CHECK) {
                const double Cn = (double)a.c_ref + (double)cp;
                const double dc = (double)cp - (double)a.fld_c[k];
                acc[SUM_DC2] += dc * dc;
                acc[SUM_C2] += Cn * Cn;
                acc[SUM_C] += Cn;
                if (L & (1u << LK::SINK)) acc[SUM_CURRENT] += (double)a.k_sink * Cn;
                if (!isfinite(cp)) acc[SUM_BAD] += 1.0;
            }
            a.fld_c[k] = cp;
        }
    }
}

// ---- the step kernel -----------------------------------------------------------------------
// Grid: x in blocks of blockDim.x columns, blockIdx.y walks rows_per_block consecutive rows of
// the (y, z) row space.  Edge nodes (first/last layer of any axis) take the general path.
template <int DIM, typename ST, bool FLOW, bool ADE, int MODE>
__global__ void __launch_bounds__(256) lbm_step_kernel(const StepArgs<DIM, ST> a)
{
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM>;
    long long off_f[F::Q], off_a[A::Q];
#pragma unroll
    for (int i = 0; i < F::Q; ++i)
        off_f[i] = F::c(i, 0) + (long long)a.px * (F::c(i, 1) + (long long)a.ny * F::c(i, 2));
#pragma unroll
    for (int i = 0; i < A::Q; ++i)
        off_a[i] = A::c(i, 0) + (long long)a.px * (A::c(i, 1) + (long long)a.ny * A::c(i, 2));

    double acc[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = 0.0;

    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int nrows = a.ny * a.nz;
    const int r0 = blockIdx.y * a.rows_per_block;
    if (x < a.nx) {
        const bool xedge = (x == 0) || (x == a.nx - 1);
        for (int rr = 0; rr < a.rows_per_block; ++rr) {
            const int r = r0 + rr;
            if (r >= nrows) break;
            const int y = r % a.ny, z = r / a.ny;
            const bool edge = xedge || y == 0 || y == a.ny - 1 ||
                              (DIM == 3 && (z == 0 || z == a.nz - 1));
            if (edge)
                update_node<DIM, ST, FLOW, ADE, MODE, true>(a, x, y, z, off_f, off_a, acc);
            else
                update_node<DIM, ST, FLOW, ADE, MODE, false>(a, x, y, z, off_f, off_a, acc);
        }
    }
    if (MODE == MODE_CHECK) block_partials(acc, a.partials);
}

// ---- argument blocks of the geometry, conversion and biofilm kernels -------------------------

struct MaskArgs {
    int nx, ny, nz, px;
    long long plane;
    int bc[3];
    const uint8_t *cls_new;  // dense node classes (x fastest, no pitch)
    const uint8_t *cls_old;  // classes before this call (ignored when reset)
    int reset;
    void *link;              // link words (pitched)
    void *fpop;              // flow populations to (re)initialise: the buffer read next
    void *gpop;              // transport populations, same
    int half;                // populations stored as FP16
    float *fld_rho, *fld_u, *fld_c;
    float c_ref;
    unsigned long long *counts;  // [0] flow-open nodes, [1] transport-open nodes
};

struct ConvArgs {
    int nx, ny, nz, px, dim;
    long long plane;
    const void *link;
    int link32;          // link words are 32-bit (3-D) or 16-bit (2-D)
    int flow_self, ade_self;
    const float *fld_rho, *fld_u, *fld_c;
    float c_ref;
    double *rho, *u, *c;  // dense outputs (device staging), each may be null
};

struct PopArgs {
    int nx, ny, nz, px;
    long long plane;
    int q;
    const void *link;
    int link32, self_bit;
    void *pop;           // pitched deviations
    int half;
    float w[19];         // weights of the set
    float offset;        // absolute = deviation + w_i * offset
    double *dense;       // q * N dense doubles
    int to_dense;        // 1: pop -> dense, 0: dense -> pop
};

struct GrowArgs {
    int nx, ny, nz, px;
    const uint8_t *cls;   // classes before the pass
    uint8_t *cls_out;     // classes after the pass
    const float *fld_c;   // C - c_ref (pitched)
    float c_ref;
    double c_thresh;
    uint64_t seed, cycle, lim;  // convert when (h >> 11) < lim = floor(prob * 2^53)
    unsigned long long *count;
};

}  // namespace mfc
