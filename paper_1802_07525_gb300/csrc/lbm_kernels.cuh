// Fused pull-scheme stream-collide kernels of the coupled flow + substrate lattice Boltzmann
// solvers (Tsompanas et al., arXiv 1802.07525, Sec. 3.1) and their residual/current reductions.
//
// Flow (Eq. 4 with the equilibrium of Eq. 5, moments Eqs. 9-10): the populations arriving at a
// node are gathered from x - c_i in the previous buffer (pull), or, where the link mask says the
// source is a wall or a blocked node, taken from the node's own opposite population (half-way
// bounce-back, Eq. 11); then BGK relaxation.  Transport (Eq. 12, moment Eq. 13): the same gather
// on D2Q5 / D3Q7 with zero-flux bounce-back, relaxation to w_i C (1 + c_i.u / cs^2) and the
// consumption w_i k C on sink nodes.
//
// Layout.  Every population plane, link word and field uses one pitched layout with a ghost
// layer around the lattice: node (x, y, z), x in [-1, nx], y in [-1, ny], z in [-1, nz] (3-D),
// sits at row0 + z*zs + y*px + x.  The row pitch px (>= nx + 2) keeps the left ghost of a row in
// the padding of the row before it, so every pull is a literal, in-bounds address and the
// interior needs no boundary branches.  Periodic axes, the moving-wall inlet and the outlet are
// realised by the boundary nodes writing, after their collision, the values their readers must
// see into the ghost cells of the buffer the next step reads; only blocks that touch such a
// boundary look at it.
//
// Threads.  One thread per node; the grid is (row / block, ny, nz), so no index needs a
// division.  Each thread issues all its loads up front: the regular pull of every direction and
// the own opposite population (bounce-back) unconditionally, selected by the link bits, so no
// load waits on another.  Every node of a row is stored, blocked ones with their zeros, so the
// stores cover whole 32-byte sectors.
//
// Precision.  Flow populations are stored as deviations from rest (f_i - w_i), transport ones
// as g_i - w_i c_ref; FP32 or FP16 storage with FP32 arithmetic, or FP64 storage with FP64
// arithmetic (Arith<ST>::T).  The rest population of each lattice
// is written as the conserved total (rho - 1, or C - kC) minus the stored moving populations, so
// rounding cannot drift mass or substrate.  Check steps accumulate residual, mass, substrate and
// current sums: per node and over a warp in FP32, over warps, blocks and the lattice in FP64 (one
// partial per block, added in a fixed order by a single-block kernel).
#pragma once

#include "lbm_lattice.cuh"

namespace mfc {

enum : int { MODE_PLAIN = 0, MODE_WRITE = 1, MODE_CHECK = 2 };

// Pitched layout with a ghost layer (see the file comment).
struct Geo {
    int nx, ny, nz;   // lattice size (nz = 1 in 2-D)
    int px;           // row pitch in elements
    long long zs;     // elements per z slab = (ny + 2) * px
    long long row0;   // element of node (0, 0, 0)
    long long plane;  // elements per population plane
    __host__ __device__ __forceinline__ long long at(int x, int y, int z) const
    {
        return row0 + (long long)z * zs + (long long)y * px + x;
    }
};

template <int DIM, typename ST, int AQ = default_aq<DIM>()> struct StepArgs {
    static constexpr int QF = FlowSet<DIM>::Q;
    static constexpr int QA = AdeSet<DIM, AQ>::Q;
    using LinkT = typename Links<DIM, AQ>::T;
    using R = typename Arith<ST>::T;  // arithmetic, field and parameter type

    Geo geo;
    int bc[3];            // boundary kind per axis
    const ST *fsrc;       // flow populations, previous step, QF planes
    ST *fdst;             // flow populations, this step
    const ST *gsrc;       // transport populations, previous step, QA planes
    ST *gdst;             // transport populations, this step
    const LinkT *link;    // link mask per node
    R *fld_rho;           // rho - 1 (written on WRITE/CHECK steps)
    R *fld_u;             // DIM planes of velocity (read by frozen-velocity transport)
    R *fld_c;             // C - c_ref
    double *partials;     // NSUM doubles per block (CHECK steps)
    R omega;              // 1 / tau
    R omega_c;            // 1 / tau_c
    R k_sink;             // consumption rate per unit concentration (low-concentration slope)
    R k_half;             // half-saturation concentration K_s of Eq. 16 (0: first order)
    R u_scale;            // factor on the velocity seen by transport
    R rho_out;            // outlet density
    R c_ref;              // offset of the stored transport populations
    int ade_dirichlet;    // transport outlet: 0 zero-gradient, 1 Dirichlet
    int cut[2];           // the low / high face of the flow axis is a cut to a neighbouring slab
    unsigned long long *bounds_err;  // checking builds: the first out-of-range element offset
    R bb_in[QF];          // moving-wall inlet term 2 w_i rho_in (c_i . u_in) / cs^2
    R gin_dev[QA];        // inlet ghost: w_i c_in (1 + c_i . u_in / cs^2) - w_i c_ref
    R gout_dev[QA];       // Dirichlet outlet ghost at c_out, same form
};

template <typename ST> using ArithT = typename Arith<ST>::T;

template <int DIM> __host__ __device__ constexpr int flow_axis() { return DIM == 2 ? 0 : 2; }

// Checking builds (MFC_CHECK_BOUNDS) test every element offset the step forms against the size
// of the array it addresses; the first offset out of range is recorded (site and offset) and the
// access goes to element 0, which lies in front of every node and ghost cell and is never read as
// a population, so nothing outside the arrays is touched and the kernel runs on.  The library
// reports the record as an error at its next synchronising call.  Other builds check nothing.
#ifdef MFC_CHECK_BOUNDS
template <typename IX>
__device__ __forceinline__ IX bound_idx(IX idx, long long limit, unsigned long long *err, int site)
{
    if ((long long)idx < 0 || (long long)idx >= limit) {
        if (err)
            atomicCAS(err, 0ull, (1ull << 63) | ((unsigned long long)site << 40) |
                                     ((unsigned long long)(long long)idx & 0xFFFFFFFFFFull));
        return (IX)0;
    }
    return idx;
}
#define MFC_IDX(idx, limit) ::mfc::bound_idx((idx), (long long)(limit), a.bounds_err, __LINE__)
#else
#define MFC_IDX(idx, limit) (idx)
#endif

// A plain (coherent) load, for values this thread stored earlier in the same kernel.
__device__ __forceinline__ float ldplain(const float *p) { return *p; }
__device__ __forceinline__ float ldplain(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ double ldplain(const double *p) { return *p; }

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum the NSUM per-node terms over the block; threads 0..NSUM-1 write them, as doubles, to
// dst[0..NSUM).  Node terms and the sums over a warp and over the block (at most 256 terms)
// are in the arithmetic type T (FP32 except in the FP64 instantiation); the sum over the blocks
// of the lattice is FP64 (finalize kernels).  GB300's FP64 rate is a small fraction of its FP32
// rate, so per-warp FP64 work would dominate an FP32 check step.
template <typename T> __device__ __forceinline__ void block_partials(T (&acc)[NSUM], double *dst)
{
    __shared__ T sh[8][NSUM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = warp_sum(acc[m]);
    if (lane == 0) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) sh[warp][m] = acc[m];
    }
    __syncthreads();
    if (threadIdx.x < NSUM) {
        T v = 0;
        for (int w = 0; w < nwarp; ++w) v += sh[w][threadIdx.x];
        dst[threadIdx.x] = (double)v;
    }
}

// FP64 sum of NSUM values per thread over a block of at most 256 threads (a multiple of 32);
// threads 0..NSUM-1 write the totals to out[0..NSUM).
__device__ __forceinline__ void block_sum_fp64(double (&acc)[NSUM], double *out)
{
    __shared__ double sh[8][NSUM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = warp_sum(acc[m]);
    if (lane == 0) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) sh[warp][m] = acc[m];
    }
    __syncthreads();
    if (threadIdx.x < NSUM) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
        out[threadIdx.x] = v;
    }
}

// ---- ghost writes ----------------------------------------------------------------------------
// After its collision, a node p on a periodic or inlet/outlet boundary writes into the ghost
// cells the values that the nodes pulling through them must receive next step:
//   periodic axis: its own post-collision population i into every periodic image q of p in the
//     ghost layer from which an interior node pulls along c_i;
//   inlet (flow): for each c_i entering the lattice, the moving-wall bounce-back value
//     F*_opp(i)(p) + bb_in[i] into q = p - c_i, which p itself pulls next step;
//     (transport): the inlet equilibrium ghost value;
//   outlet: for each c_i leaving the outlet ghost layer inwards, the value of the last-layer
//     source p (flow: equilibrium at rho_out with p's velocity; transport: p's own population,
//     or the Dirichlet ghost value) into q = p + e_flow and its periodic images.
// Each ghost value has exactly one reader and one writer.

template <int DIM>
__device__ __forceinline__ bool interior(const Geo &g, int x, int y, int z)
{
    return x >= 0 && x < g.nx && y >= 0 && y < g.ny && (DIM == 2 || (z >= 0 && z < g.nz));
}

// Does node p have to write any ghost value?
template <int DIM>
__device__ __forceinline__ bool on_open_boundary(const Geo &g, const int (&bc)[3], int x, int y, int z)
{
    bool b = (bc[0] != BC_WALL) && (x == 0 || x == g.nx - 1);
    b = b || ((bc[1] != BC_WALL) && (y == 0 || y == g.ny - 1));
    if (DIM == 3) b = b || ((bc[2] != BC_WALL) && (z == 0 || z == g.nz - 1));
    return b;
}

// Write v into ghost cells q = b + s of plane i, over the periodic image shifts s of base cell
// b (the zero shift too when include_zero), wherever an interior node pulls q along c_i.  With
// `lazy`, v is read from there, and only when some image is written (a node on no periodic
// boundary reads nothing).
template <int DIM, typename SET, typename ST>
__device__ __forceinline__ void ghost_images(const Geo &g, const int (&bc)[3], ST *pop, int i,
                                             int bx, int by, int bz, bool include_zero,
                                             ArithT<ST> v, const ST *lazy = nullptr)
{
    const int n[3] = {g.nx, g.ny, g.nz};
    const int b[3] = {bx, by, bz};
    int opts[3][3];
    int nopt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        nopt[a] = 1;
        opts[a][0] = 0;
        opts[a][1] = 0;
        opts[a][2] = 0;
        if (a < DIM && bc[a] == BC_PERIODIC) {
            if (b[a] == 0) opts[a][nopt[a]++] = n[a];
            if (b[a] == n[a] - 1) opts[a][nopt[a]++] = -n[a];
        }
    }
    if (lazy) {
        if (!include_zero && nopt[0] * nopt[1] * nopt[2] == 1) return;  // no image to write
        v = ldplain(lazy);
    }
    for (int ix = 0; ix < nopt[0]; ++ix)
        for (int iy = 0; iy < nopt[1]; ++iy)
            for (int iz = 0; iz < nopt[2]; ++iz) {
                if (!include_zero && ix == 0 && iy == 0 && iz == 0) continue;
                const int q0 = b[0] + opts[0][ix], q1 = b[1] + opts[1][iy], q2 = b[2] + opts[2][iz];
                if (!interior<DIM>(g, q0 + SET::c(i, 0), q1 + SET::c(i, 1), q2 + SET::c(i, 2))) continue;
                st(pop + (long long)i * g.plane + g.at(q0, q1, q2), v);
            }
}

// Whether ghost writes read a node's post-collision populations back only where a ghost value
// needs them (measured 4-6% faster for FP16 2-D steps), or all of them up front (FP32 2-D steps,
// whose 32-register budget spills in the hot loop with the lazy form).
template <int DIM, typename ST> struct LazyGhosts {
    static constexpr bool value = !(DIM == 2 && sizeof(ST) == 4);
};

// Flow ghost writes of node p (stored at k) with velocity (u0, u1, u2) and link word L; the
// node's post-collision populations are read back from pop, where this thread just stored them.
template <int DIM, typename ST, int AQ>
__device__ __forceinline__ void flow_ghosts(const StepArgs<DIM, ST, AQ> &a, ST *pop, int x, int y, int z,
                                         long long k, uint32_t L, ArithT<ST> u0, ArithT<ST> u1, ArithT<ST> u2)
{
    using R = ArithT<ST>;
    using F = FlowSet<DIM>;
    constexpr int FA = flow_axis<DIM>();
    const int p[3] = {x, y, z};
    const int n[3] = {a.geo.nx, a.geo.ny, a.geo.nz};
    const bool inout = a.bc[FA] == BC_INOUT;
    const R uv[3] = {u0, u1, DIM == 3 ? u2 : R(0)};
    const R uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
#pragma unroll
    for (int i = 1; i < F::Q; ++i) {
        if (LazyGhosts<DIM, ST>::value) {
            ghost_images<DIM, F, ST>(a.geo, a.bc, pop, i, x, y, z, false, R(0), pop + (long long)i * a.geo.plane + k);
        } else {
            const R di = ldplain(pop + (long long)i * a.geo.plane + k);
            ghost_images<DIM, F, ST>(a.geo, a.bc, pop, i, x, y, z, false, di);
        }
        if (!inout) continue;
        const int cf = F::c(i, FA);
        if (p[FA] == 0 && cf == 1 && !a.cut[0] && !((L >> i) & 1u)) {  // inlet: the node's own next-step pull
            const int q0 = x - F::c(i, 0), q1 = y - F::c(i, 1), q2 = z - F::c(i, 2);
            st(pop + MFC_IDX((long long)i * a.geo.plane + a.geo.at(q0, q1, q2), F::Q * a.geo.plane),
               ldplain(pop + MFC_IDX((long long)F::opp(i) * a.geo.plane + k, F::Q * a.geo.plane)) + a.bb_in[i]);
        }
        if (p[FA] == n[FA] - 1 && cf == -1 && !a.cut[1]) {  // outlet ghost fed by this last-layer node
            const R cu = F::c(i, 0) * uv[0] + F::c(i, 1) * uv[1] + F::c(i, 2) * uv[2];
            const R v = weight<F, R>(i) * (a.rho_out - R(1) +
                                       a.rho_out * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
            int b[3] = {x, y, z};
            b[FA] = n[FA];
            ghost_images<DIM, F, ST>(a.geo, a.bc, pop, i, b[0], b[1], b[2], true, v);
        }
    }
}

// Transport ghost writes of node p (stored at k) with link word L; the node's post-collision
// populations are read back from pop.
template <int DIM, typename ST, int AQ>
__device__ __forceinline__ void ade_ghosts(const StepArgs<DIM, ST, AQ> &a, ST *pop, int x, int y, int z,
                                        long long k, uint32_t L)
{
    using R = ArithT<ST>;
    using A = AdeSet<DIM, AQ>;
    constexpr int FA = flow_axis<DIM>();
    const int p[3] = {x, y, z};
    const int n[3] = {a.geo.nx, a.geo.ny, a.geo.nz};
    const bool inout = a.bc[FA] == BC_INOUT;
    // Eager form: every read-back is issued before the first ghost store, so the loads overlap
    // (a load placed after a store that may alias it cannot be moved ahead of it).  Measured on
    // the FP32 2-D step: 42.8 against 44.5 us per 2048x1024 step.  The same change in
    // flow_ghosts spills at 32 registers and runs slower.
    R ev[A::Q];
#pragma unroll
    for (int i = 1; i < A::Q; ++i)
        ev[i] = LazyGhosts<DIM, ST>::value ? R(0) : ldplain(pop + (long long)i * a.geo.plane + k);
#pragma unroll
    for (int i = 1; i < A::Q; ++i) {
        const ST *own = pop + (long long)i * a.geo.plane + k;
        const R ei = ev[i];
        ghost_images<DIM, A, ST>(a.geo, a.bc, pop, i, x, y, z, false, ei, LazyGhosts<DIM, ST>::value ? own : nullptr);
        if (!inout) continue;
        const int cf = A::c(i, FA);
        if (p[FA] == 0 && cf == 1 && !a.cut[0] && !((L >> (Links<DIM, AQ>::ADE_SELF + i)) & 1u)) {
            const int q0 = x - A::c(i, 0), q1 = y - A::c(i, 1), q2 = z - A::c(i, 2);
            st(pop + MFC_IDX((long long)i * a.geo.plane + a.geo.at(q0, q1, q2), A::Q * a.geo.plane), a.gin_dev[i]);
        }
        if (p[FA] == n[FA] - 1 && cf == -1 && !a.cut[1]) {
            int b[3] = {x, y, z};
            b[FA] = n[FA];
            if (a.ade_dirichlet) ghost_images<DIM, A, ST>(a.geo, a.bc, pop, i, b[0], b[1], b[2], true, a.gout_dev[i]);
            else ghost_images<DIM, A, ST>(a.geo, a.bc, pop, i, b[0], b[1], b[2], true, ei,
                                          LazyGhosts<DIM, ST>::value ? own : nullptr);
        }
    }
}

// During a step the inlet and the transport outlet need no ghost values: a node on the inlet
// takes its inlet populations itself when it gathers (the moving-wall bounce-back value
// F*_opp(i) + bb_in[i] from its own previous populations; the transport inlet value), and so
// does a transport node on the outlet (its own previous population of the same direction, or the
// Dirichlet value).  What remains for the step to write: the periodic images of boundary nodes,
// and the flow outlet values (an equilibrium from the last layer's velocity, pulled along the
// diagonals by the neighbouring rows too).  The functions above write every ghost value, for
// the state set from outside a step.

template <int DIM>
__device__ __forceinline__ bool on_periodic_boundary(const Geo &g, const int (&bc)[3], int x, int y, int z)
{
    bool b = (bc[0] == BC_PERIODIC) && (x == 0 || x == g.nx - 1);
    b = b || ((bc[1] == BC_PERIODIC) && (y == 0 || y == g.ny - 1));
    if (DIM == 3) b = b || ((bc[2] == BC_PERIODIC) && (z == 0 || z == g.nz - 1));
    return b;
}

// Does node p write ghost values during a flow step (periodic images, flow outlet values)?
template <int DIM>
__device__ __forceinline__ bool step_writes_ghosts(const Geo &g, const int (&bc)[3], int x, int y, int z)
{
    constexpr int FA = flow_axis<DIM>();
    const int pf = FA == 0 ? x : z, nf = FA == 0 ? g.nx : g.nz;
    return on_periodic_boundary<DIM>(g, bc, x, y, z) || (bc[FA] == BC_INOUT && pf == nf - 1);
}

// Flow ghost writes of a step: the periodic images of node p (its post-collision populations
// read back from pop, where this thread just stored them) and, on the last layer of the
// inlet/outlet axis, the outlet values from its velocity.
template <int DIM, typename ST, int AQ>
__device__ __forceinline__ void flow_ghosts_step(const StepArgs<DIM, ST, AQ> &a, ST *pop, int x, int y, int z,
                                                 long long k, ArithT<ST> u0, ArithT<ST> u1, ArithT<ST> u2)
{
    using R = ArithT<ST>;
    using F = FlowSet<DIM>;
    constexpr int FA = flow_axis<DIM>();
    const int p[3] = {x, y, z};
    const int n[3] = {a.geo.nx, a.geo.ny, a.geo.nz};
    if (on_periodic_boundary<DIM>(a.geo, a.bc, x, y, z)) {
#pragma unroll
        for (int i = 1; i < F::Q; ++i) {
            const R di = ldplain(pop + (long long)i * a.geo.plane + k);
            ghost_images<DIM, F, ST>(a.geo, a.bc, pop, i, x, y, z, false, di);
        }
    }
    if (a.bc[FA] == BC_INOUT && p[FA] == n[FA] - 1 && !a.cut[1]) {
        const R uv[3] = {u0, u1, DIM == 3 ? u2 : R(0)};
        const R uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
#pragma unroll
        for (int i = 1; i < F::Q; ++i) {
            if (F::c(i, FA) != -1) continue;
            const R cu = F::c(i, 0) * uv[0] + F::c(i, 1) * uv[1] + F::c(i, 2) * uv[2];
            const R v = weight<F, R>(i) * (a.rho_out - R(1) +
                                       a.rho_out * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
            int b[3] = {x, y, z};
            b[FA] = n[FA];
            ghost_images<DIM, F, ST>(a.geo, a.bc, pop, i, b[0], b[1], b[2], true, v);
        }
    }
}

// Transport ghost writes of a step: the periodic images of node p.
template <int DIM, typename ST, int AQ>
__device__ __forceinline__ void ade_ghosts_step(const StepArgs<DIM, ST, AQ> &a, ST *pop, int x, int y, int z,
                                                long long k)
{
    using R = ArithT<ST>;
    using A = AdeSet<DIM, AQ>;
    if (!on_periodic_boundary<DIM>(a.geo, a.bc, x, y, z)) return;
#pragma unroll
    for (int i = 1; i < A::Q; ++i) {
        const R ei = ldplain(pop + (long long)i * a.geo.plane + k);
        ghost_images<DIM, A, ST>(a.geo, a.bc, pop, i, x, y, z, false, ei);
    }
}

// ---- the step kernel -------------------------------------------------------------------------

// Does the tile of n nodes from (x0, y, z) along x hold a node that writes ghost values during a
// step, or takes inlet/outlet values when it gathers?
template <int DIM>
__device__ __forceinline__ bool tile_on_open_boundary(const Geo &g, const int (&bc)[3], int x0, int n, int y, int z)
{
    bool b = bc[0] != BC_WALL && (x0 == 0 || x0 + n >= g.nx);
    b = b || (bc[1] != BC_WALL && (y == 0 || y == g.ny - 1));
    if (DIM == 3) b = b || (bc[2] != BC_WALL && (z == 0 || z == g.nz - 1));
    return b;
}

// Register caps of the step kernels: 2-D FP32 plain steps fit 32 registers (8 blocks of 256
// threads per SM); 2-D FP16 plain steps (their conversions need more registers: 8% faster at 40
// than at 32), FP32 2-D steps with D2Q9 transport, and 2-D store/check steps 40.  3-D steps are
// latency-bound and gain from warps: FP32 with 5 blocks of 256 threads (51 registers: 148 us per
// 256x128x128 step, against 211 us uncapped at 128 registers) and FP16 with 4 (64 registers:
// 154 against 178 us); tighter caps spill and run slower.  With 32-bit offsets the FP16 3-D plain
// step fits 48 registers without spills, and 5 blocks run it 6% faster (119.0 against 126.8 us);
// the FP32 3-D one gains nothing from 6 blocks (138.9 against 139.5 us, with spills).  The FP64
// instantiation (a parity reference, twice the registers per value) gets 128.
template <int DIM, int MODE, typename ST = float, int AQ = default_aq<DIM>(), bool IDX32 = false>
struct StepOccupancy {
    static constexpr int blocks =
        (IDX32 && MODE == MODE_PLAIN && DIM == 3 && sizeof(ST) == 2) ? 5 :
        sizeof(ST) == 8 ? 2
                        : (DIM == 2 ? ((MODE == MODE_PLAIN && sizeof(ST) == 4 && AQ == 5) ? 8 : 6)
                                    : (sizeof(ST) == 4 ? 5 : 4));
};

// Two equivalent ways to realise the open boundaries in a step, chosen per kernel by measurement:
//   B_WRITER: one code path; boundary nodes write every ghost value after their collision,
//     including the inlet and transport-outlet values that they themselves pull next step.
//   B_BOUNDARY / B_INTERIOR: reader side; a node on the inlet (outlet) takes those values itself
//     when it gathers, boundary nodes write only periodic images and the flow outlet values, and
//     tiles that touch no open boundary run a second code path with no boundary handling at all.
// Measured on GB300: the reader-side form makes the batch step 20% and the FP16 2-D step 6-7%
// faster; the FP32 2-D step (32 registers) runs faster in the writer form.  All steps of one
// lattice must take the same form: a writer-side step pulls inlet and transport-outlet values
// from ghost cells that only a writer-side step before it fills.  FP16 storage takes the reader
// form in 2-D and 3-D, because its plain steps (two rows per thread) are fastest in it; its
// single-node steps (check, stored-field and 64-bit-offset steps) follow.
enum : int { B_WRITER = 0, B_BOUNDARY = 1, B_INTERIOR = 2 };
template <int DIM, typename ST, int AQ = default_aq<DIM>()> struct ReaderBoundaries {
    // the single-lattice step kernel; D2Q9 transport keeps writer-side ghosts, whose outlet
    // values along the diagonals come from the neighbouring row
    static constexpr bool step = sizeof(ST) == 2 && AQ == default_aq<DIM>();
};

// One step of node (x0 + threadIdx.x, y, z) of one lattice, in a tile of blockDim.x nodes from
// (x0, y, z).  Threads with x >= nx return at once, except in check steps, where they compute on
// a copy of the last node of the row, store nothing and add nothing, so that the whole block
// joins the reduction.  acc receives the node's check-step terms.  BFORM: the boundary form
// (B_BOUNDARY and B_INTERIOR are for tiles that do / do not touch an open boundary).
// The consumption law of a kernel: first order (k C), the saturating substrate factor of
// Eq. 16 (k C K_s / (K_s + C)), or chosen per instance at run time from k_half (batch kernels,
// whose instances may differ).  Single-lattice step kernels are instantiated per law, so that
// the first-order kernels carry no code for the other.
enum : int { SINK_LINEAR = 0, SINK_MONOD = 1, SINK_RUNTIME = 2 };

// IX: the integer type of the element offsets: long long, or int where every population array
// has fewer than 2^31 elements (one IMAD.WIDE per address instead of 64-bit offset arithmetic).
template <int DIM, typename ST, bool FLOW, bool ADE, int MODE, int BFORM, int AQ, int SINK = SINK_RUNTIME,
          typename IX = long long>
__device__ __forceinline__ void step_node(const StepArgs<DIM, ST, AQ> &a, int x0, int y, int z, ArithT<ST> (&acc)[NSUM])
{
    using R = ArithT<ST>;
    static_assert(BFORM == B_WRITER || AdeSet<DIM, AQ>::Q == default_aq<DIM>(),
                  "reader-side boundaries take the transport outlet from the node itself: axis-aligned sets only");
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM, AQ>;
    using LK = Links<DIM, AQ>;
    const Geo g = a.geo;
    const int x = x0 + threadIdx.x;
    if (MODE != MODE_CHECK && x >= g.nx) return;
    const bool valid = MODE != MODE_CHECK || x < g.nx;
    const IX k = (IX)g.row0 + (IX)z * (IX)g.zs + (IX)y * (IX)g.px + (IX)(x < g.nx ? x : g.nx - 1);
    const IX P = (IX)g.plane;
    const uint32_t L = __ldg(a.link + MFC_IDX(k, P));
    constexpr bool READER = BFORM != B_WRITER;
    const bool bnd_tile = BFORM == B_WRITER ? tile_on_open_boundary<DIM>(g, a.bc, x0, blockDim.x, y, z)
                                            : BFORM == B_BOUNDARY;
    const bool ghosts = bnd_tile && valid &&
                        (READER ? step_writes_ghosts<DIM>(g, a.bc, x, y, z) : on_open_boundary<DIM>(g, a.bc, x, y, z));
    // reader side: on the inlet / outlet layer of an inlet/outlet axis (the node takes those
    // values itself)
    constexpr int FA = flow_axis<DIM>();
    const int pf = FA == 0 ? x : z;
    const bool inout = READER && bnd_tile && a.bc[FA] == BC_INOUT;
    const bool at_in = inout && pf == 0 && !a.cut[0];
    const bool at_out = inout && pf == (FA == 0 ? g.nx : g.nz) - 1 && !a.cut[1];
    // How a bounce-back population is fetched.  Unconditional own-opposite loads, selected
    // afterwards, keep every load independent of the link word; one load per direction from an
    // address chosen by the link bit halves the load instructions.  With 64-bit offsets the
    // selection costs more than it saves in 2-D (measured slower in FP32 and FP16), and pays in
    // 3-D (19 + 7 directions under tight register caps: 4% faster in FP32, 3% in FP16); with
    // 32-bit offsets the choice is one 32-bit select, and it pays in 2-D too (2048x1024 FP32
    // 45.1 -> 43.5 us, 4096x1024 FP16 65.5 -> 61.4 us).
    constexpr bool SELECT_LOADS = DIM == 3 || sizeof(IX) == 4;
    R u[3] = {R(0), R(0), R(0)};
    // check step: the previous fields of this node (read before this thread overwrites them),
    // issued first so that their latency overlaps the population loads
    R u_prev[3] = {R(0), R(0), R(0)}, c_prev = R(0);
    if (MODE == MODE_CHECK) {
        if (FLOW) {
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) u_prev[ax] = ldplain(a.fld_u + MFC_IDX(ax * g.plane + k, DIM * P));
        }
        if (ADE) c_prev = ldplain(a.fld_c + MFC_IDX(k, P));
    }

    if (FLOW) {
        R d[F::Q];
#pragma unroll
        for (int i = 0; i < F::Q; ++i) {
            const IX off = (IX)F::c(i, 0) + (IX)F::c(i, 1) * (IX)g.px + (IX)F::c(i, 2) * (IX)g.zs;
            // inlet link (entering across the inlet, no wall in between): moving-wall bounce-back
            const bool bb = i > 0 && ((L >> i) & 1u);
            const bool inj = F::c(i, FA) == 1 && at_in && !bb;
            if (SELECT_LOADS) {
                const IX o = (bb || inj) ? (IX)F::opp(i) * P : (IX)i * P - off;
                d[i] = ld(a.fsrc + MFC_IDX(k + o, F::Q * P));
                if (F::c(i, FA) == 1 && inj) d[i] += a.bb_in[i];
            } else {
                const R src = ld(a.fsrc + MFC_IDX((IX)i * P + k - off, F::Q * P));
                if (i == 0) {
                    d[0] = src;
                } else {
                    const R own = ld(a.fsrc + MFC_IDX((IX)F::opp(i) * P + k, F::Q * P));
                    d[i] = bb ? own : src;
                    if (F::c(i, FA) == 1 && inj) d[i] = own + a.bb_in[i];
                }
            }
        }
        const bool open = !(L & (1u << LK::FLOW_SELF));
        R rp = R(0), j[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int i = 0; i < F::Q; ++i) {
            if (!open) d[i] = R(0);  // blocked nodes hold no populations
            rp += d[i];
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) j[ax] += F::c(i, ax) * d[i];
        }
        const R inv = recip(R(1) + rp);  // FP32: fast reciprocal, <= 2 ulp
        R uu = R(0);
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) {
            u[ax] = j[ax] * inv;
            uu += u[ax] * u[ax];
        }
        // BGK relaxation of the moving populations, then the rest one closes the mass
        R moved = R(0);
#pragma unroll
        for (int i = 1; i < F::Q; ++i) {
            R cu = R(0);
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) cu += F::c(i, ax) * u[ax];
            const R feq = weight<F, R>(i) * (rp + (R(1) + rp) * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
            const R v = kept(a.fdst, d[i] + a.omega * (feq - d[i]));
            moved += v;
            if (valid) st(a.fdst + MFC_IDX((IX)i * P + k, F::Q * P), v);
        }
        if (valid) st(a.fdst + MFC_IDX(k, F::Q * P), rp - moved);
        if (ghosts && open) {
            if constexpr (READER) flow_ghosts_step<DIM, ST>(a, a.fdst, x, y, z, k, u[0], u[1], u[2]);
            else flow_ghosts<DIM, ST>(a, a.fdst, x, y, z, k, L, u[0], u[1], u[2]);
        }
        if (MODE != MODE_PLAIN && valid) {
            if (MODE == MODE_CHECK && open) {
                R du2 = R(0), u2 = R(0);
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) {
                    const R dd = u[ax] - u_prev[ax];  // exact for nearby values
                    du2 += dd * dd;
                    u2 += u[ax] * u[ax];
                }
                acc[SUM_DU2] = du2;
                acc[SUM_U2] = u2;
                acc[SUM_MASS] = R(1) + rp;
                if (!isfinite(rp) || !isfinite(u2)) acc[SUM_BAD] = R(1);
                // the BGK equilibrium is a low-Mach expansion: at or past the sound speed, or at a
                // non-positive density, the solve has left the scheme's range
                if (R(3) * u2 >= R(1) || rp <= R(-1)) acc[SUM_FAST] = R(1);
            }
            a.fld_rho[MFC_IDX(k, P)] = rp;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) a.fld_u[MFC_IDX(ax * g.plane + k, DIM * P)] = u[ax];
        }
    }

    if (ADE) {
        if (FLOW) {
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) u[ax] *= a.u_scale;  // 0 on flow-blocked nodes
        } else if (!(L & (1u << LK::FLOW_SELF))) {
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) u[ax] = a.fld_u[MFC_IDX(ax * g.plane + k, DIM * P)] * a.u_scale;
        }
        R e[A::Q];
#pragma unroll
        for (int i = 0; i < A::Q; ++i) {
            const IX off = (IX)A::c(i, 0) + (IX)A::c(i, 1) * (IX)g.px + (IX)A::c(i, 2) * (IX)g.zs;
            // inlet value; at the outlet, zero gradient (the node's own previous population of the
            // same direction) or the Dirichlet value
            const bool bb = i > 0 && ((L >> (LK::ADE_SELF + i)) & 1u);
            const bool in_v = A::c(i, FA) == 1 && at_in && !bb;
            const bool out_v = A::c(i, FA) == -1 && at_out && !bb;
            if (SELECT_LOADS) {
                const IX o = bb ? (IX)A::opp(i) * P : (IX)i * P - (out_v ? (IX)0 : off);
                e[i] = ld(a.gsrc + MFC_IDX(k + o, A::Q * P));
            } else {
                const R src = ld(a.gsrc + MFC_IDX((IX)i * P + k - off, A::Q * P));
                if (i == 0) {
                    e[0] = src;
                } else {
                    const R own = ld(a.gsrc + MFC_IDX((IX)A::opp(i) * P + k, A::Q * P));
                    e[i] = bb ? own : src;
                    if (A::c(i, FA) == -1 && out_v) e[i] = ld(a.gsrc + MFC_IDX((IX)i * P + k, A::Q * P));
                }
            }
            if (A::c(i, FA) == 1 && in_v) e[i] = a.gin_dev[i];
            if (A::c(i, FA) == -1 && out_v && a.ade_dirichlet) e[i] = a.gout_dev[i];
        }
        const bool open = !(L & (1u << LK::ADE_SELF));
        R cp = R(0);
#pragma unroll
        for (int i = 0; i < A::Q; ++i) {
            if (!open) e[i] = R(0);
            cp += e[i];
        }
        // consumption (Eq. 16's substrate factor): k C, or k C K_s / (K_s + C)
        R sink = R(0);
        if constexpr (SINK == SINK_LINEAR) {
            sink = (L & (1u << LK::SINK)) ? a.k_sink * (a.c_ref + cp) : R(0);
        } else if (L & (1u << LK::SINK)) {
            const R Cs = a.c_ref + cp;
            sink = a.k_sink * Cs;
            if (SINK == SINK_MONOD || a.k_half > R(0)) sink = sink * a.k_half * recip(a.k_half + Cs);
        }
        R uu_ade = R(0);
        if (A::quadratic) {
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) uu_ade += u[ax] * u[ax];
        }
        R moved = R(0);
#pragma unroll
        for (int i = 1; i < A::Q; ++i) {
            R cu = R(0);
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) cu += A::c(i, ax) * u[ax];
            // linear (D2Q5 / D3Q7) or the quadratic equilibrium of Eq. 5 (D2Q9), as deviations
            const R shape = A::quadratic ? 3.0f * cu + 4.5f * cu * cu - 1.5f * uu_ade : cu * A::inv_cs2;
            const R geq = weight<A, R>(i) * (cp + (a.c_ref + cp) * shape);
            const R v = kept(a.gdst, e[i] + a.omega_c * (geq - e[i]) - weight<A, R>(i) * sink);
            moved += v;
            if (valid) st(a.gdst + MFC_IDX((IX)i * P + k, A::Q * P), v);
        }
        if (valid) st(a.gdst + MFC_IDX(k, A::Q * P), cp - sink - moved);
        if (ghosts && open) {
            if constexpr (READER) ade_ghosts_step<DIM, ST>(a, a.gdst, x, y, z, k);
            else ade_ghosts<DIM, ST>(a, a.gdst, x, y, z, k, L);
        }
        if (MODE != MODE_PLAIN && valid) {
            if (MODE == MODE_CHECK && open) {
                const R Cn = a.c_ref + cp;
                const R dc = cp - c_prev;
                acc[SUM_DC2] = dc * dc;
                acc[SUM_C2] = Cn * Cn;
                acc[SUM_C] = Cn;
                if constexpr (SINK == SINK_LINEAR) {
                    if (L & (1u << LK::SINK)) acc[SUM_CURRENT] = a.k_sink * Cn;
                } else {
                    acc[SUM_CURRENT] = sink;
                }
                if (!isfinite(cp)) acc[SUM_BAD] += R(1);
            }
            a.fld_c[MFC_IDX(k, P)] = open ? cp : -a.c_ref;
        }
    }
}

// One step of one lattice: one thread per node, grid (row / block, ny, nz); one reduction
// partial per block on check steps.
template <int DIM, typename ST, bool FLOW, bool ADE, int MODE, int AQ = default_aq<DIM>(), int SINK = SINK_LINEAR,
          bool IDX32 = false>
__global__ void __launch_bounds__(256, StepOccupancy<DIM, MODE, ST, AQ, IDX32>::blocks) lbm_step_kernel(const StepArgs<DIM, ST, AQ> a)
{
    using IX = typename std::conditional<IDX32, int, long long>::type;
    using R = ArithT<ST>;
    R acc[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = R(0);
    const int x0 = blockIdx.x * blockDim.x;
    // 3-D: the last plane first (blocks are dispatched in z order), so that the outlet plane's
    // ghost work overlaps the bulk of the step instead of lengthening its tail (1.5% faster on
    // 256x128x128); 2-D keeps row order, whose locality is worth more.
    const int z = DIM == 3 ? (blockIdx.z == 0 ? (int)gridDim.z - 1 : (int)blockIdx.z - 1) : 0;
    if constexpr (ReaderBoundaries<DIM, ST, AQ>::step) {
        if (tile_on_open_boundary<DIM>(a.geo, a.bc, x0, blockDim.x, blockIdx.y, z))
            step_node<DIM, ST, FLOW, ADE, MODE, B_BOUNDARY, AQ, SINK, IX>(a, x0, blockIdx.y, z, acc);
        else
            step_node<DIM, ST, FLOW, ADE, MODE, B_INTERIOR, AQ, SINK, IX>(a, x0, blockIdx.y, z, acc);
    } else {
        step_node<DIM, ST, FLOW, ADE, MODE, B_WRITER, AQ, SINK, IX>(a, x0, blockIdx.y, z, acc);
    }
    if (MODE == MODE_CHECK)
        block_partials(acc, a.partials + ((size_t)blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y *
                                                                                  blockIdx.z)) * NSUM);
}

// ---- many lattices in one launch -------------------------------------------------------------
// A tile is one block's worth of nodes along x of one row of one lattice (instance).  The tile
// table lists the tiles of every instance of the launch, instance after instance; a fixed grid
// of blocks (a few per SM) walks it with a stride of the grid, so the launch shape does not
// depend on which instances are active.  Each instance slot holds two argument blocks, for the
// two buffer parities; a step uses the one of its parity.
struct Tile {
    int slot, x0, y, z;
};

template <int DIM, typename ST> struct BatchArgs {
    const StepArgs<DIM, ST> *inst;  // [2 * slot + parity]
    const Tile *tiles;              // tile table
    const int *ntiles;              // tiles in the table (device value, set before the launch)
    double *partials;               // NSUM per tile (check steps)
    int parity;
};

// Element offsets are 32-bit: a batch admits only instances whose population arrays have fewer
// than 2^31 elements.  The tile loop and the shared argument block take registers of their own:
// 2-D batch steps are capped at 48 registers (5 blocks of 256 threads per SM), where they do not
// spill; 3-D batch steps take the caps of the 3-D step kernel.
template <int DIM, typename ST, bool FLOW, bool ADE, int MODE>
__global__ void __launch_bounds__(256, DIM == 2 ? 5 : StepOccupancy<DIM, MODE, ST>::blocks)
    lbm_batch_kernel(const BatchArgs<DIM, ST> b)
{
    static_assert(sizeof(StepArgs<DIM, ST>) % 4 == 0, "argument block copied as 32-bit words");
    __shared__ StepArgs<DIM, ST> sa;  // arguments of the instance of the current tile
    constexpr int WORDS = (int)(sizeof(StepArgs<DIM, ST>) / 4);
    const int n = *b.ntiles;
    int cur = -1;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const Tile tile = b.tiles[t];
        if (tile.slot != cur) {  // uniform over the block: every thread reads the same entry
            __syncthreads();     // the previous instance's arguments are no longer read
            const uint32_t *src = reinterpret_cast<const uint32_t *>(b.inst + 2 * tile.slot + b.parity);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
            for (int w = threadIdx.x; w < WORDS; w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            cur = tile.slot;
        }
        ArithT<ST> acc[NSUM];
#pragma unroll
        for (int m = 0; m < NSUM; ++m) acc[m] = 0;
        constexpr int AQ = default_aq<DIM>();
        if (tile_on_open_boundary<DIM>(sa.geo, sa.bc, tile.x0, blockDim.x, tile.y, tile.z))
            step_node<DIM, ST, FLOW, ADE, MODE, B_BOUNDARY, AQ, SINK_RUNTIME, int>(sa, tile.x0, tile.y, tile.z, acc);
        else
            step_node<DIM, ST, FLOW, ADE, MODE, B_INTERIOR, AQ, SINK_RUNTIME, int>(sa, tile.x0, tile.y, tile.z, acc);
        if (MODE == MODE_CHECK) {
            block_partials(acc, b.partials + (size_t)t * NSUM);
            __syncthreads();  // the reduction's shared memory is reused by the next tile
        }
    }
}

// Per instance slot s, the sums over its tiles [range[s].x, range[s].y) of the launch, in FP64
// and in a fixed order, and the two residuals: results[s * NRESULT ...].  One block per slot.
__device__ __forceinline__ void batch_finalize_slot(const int2 range, const double *partials,
                                                    double *res)
{
    double acc[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = 0.0;
    for (int t = range.x + threadIdx.x; t < range.y; t += blockDim.x) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) acc[m] += partials[(size_t)t * NSUM + m];
    }
    __shared__ double r[NSUM];
    block_sum_fp64(acc, r);
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) res[m] = r[m];
        res[RES_FLOW] = r[SUM_U2] > 0.0 ? sqrt(r[SUM_DU2] / r[SUM_U2]) : (r[SUM_DU2] > 0.0 ? INFINITY : 0.0);
        res[RES_ADE] = r[SUM_C2] > 0.0 ? sqrt(r[SUM_DC2] / r[SUM_C2]) : (r[SUM_DC2] > 0.0 ? INFINITY : 0.0);
    }
}

// Write the ghost cells of the current buffers (a.fdst, a.gdst) from the state they hold, after
// the state was set from outside a step (geometry change, parameters, a population write).
template <int DIM, typename ST, int AQ = default_aq<DIM>()>
__global__ void fill_ghosts_kernel(const StepArgs<DIM, ST, AQ> a)
{
    using R = ArithT<ST>;
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM, AQ>;
    using LK = Links<DIM, AQ>;
    const Geo &g = a.geo;
    const long long N = (long long)g.nx * g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(q % g.nx), y = (int)((q / g.nx) % g.ny), z = (int)(q / ((long long)g.nx * g.ny));
        const long long k = g.at(x, y, z);
        const uint32_t L = a.link[k];
        if (!(L & (1u << LK::FLOW_SELF))) {
            R d[F::Q], rp = R(0), j[3] = {R(0), R(0), R(0)};
#pragma unroll
            for (int i = 0; i < F::Q; ++i) {
                d[i] = ld(a.fdst + (long long)i * g.plane + k);
                rp += d[i];
                for (int ax = 0; ax < DIM; ++ax) j[ax] += F::c(i, ax) * d[i];
            }
            R u[3] = {R(0), R(0), R(0)};
            for (int ax = 0; ax < DIM; ++ax) u[ax] = j[ax] / (R(1) + rp);
            if (on_open_boundary<DIM>(g, a.bc, x, y, z)) flow_ghosts<DIM, ST>(a, a.fdst, x, y, z, k, L, u[0], u[1], u[2]);
        }
        if (!(L & (1u << LK::ADE_SELF))) {
            R e[A::Q];
            for (int i = 0; i < A::Q; ++i) e[i] = ld(a.gdst + (long long)i * g.plane + k);
            if (on_open_boundary<DIM>(g, a.bc, x, y, z)) ade_ghosts<DIM, ST>(a, a.gdst, x, y, z, k, L);
        }
    }
}

// ---- argument blocks of the geometry, conversion and biofilm kernels -------------------------

struct MaskArgs {
    Geo geo;
    int bc[3];
    const uint8_t *cls_new;  // dense node classes (x fastest, no pitch)
    const uint8_t *cls_old;  // classes before this call (ignored when reset)
    int reset;
    void *link;              // link words (pitched)
    void *fpop;              // flow populations to (re)initialise: the buffer read next
    void *gpop;              // transport populations, same
    int half;                // populations stored as FP16
    int dbl;                 // populations and fields stored as FP64 (else fields are FP32)
    void *fld_rho, *fld_u, *fld_c;
    float c_ref;
    unsigned long long *counts;  // [0] flow-open nodes, [1] transport-open nodes
    int cut[2];                  // the low / high face of the flow axis is a cut
    const uint8_t *halo_cls[2];  // the neighbour's classes next to each cut (null: open)
};

struct ConvArgs {
    Geo geo;
    int dim;
    const void *link;
    int link32;          // link words are 32-bit (3-D) or 16-bit (2-D)
    int flow_self, ade_self;
    int dbl;             // fields stored as FP64 (else FP32)
    const void *fld_rho, *fld_u, *fld_c;
    float c_ref;
    double *rho, *u, *c;  // dense outputs (device staging), each may be null
};

struct PopArgs {
    Geo geo;
    int q;
    const void *link;
    int link32, self_bit;
    void *pop;           // pitched deviations
    int half, dbl;       // stored as FP16 / FP64 (else FP32)
    double w[19];        // weights of the set (the FP32 constants, or the FP64 ones)
    double offset;       // absolute = deviation + w_i * offset
    double *dense;       // q * N dense doubles
    int to_dense;        // 1: pop -> dense, 0: dense -> pop
};

struct GrowArgs {
    Geo geo;
    const uint8_t *cls;   // classes before the pass
    uint8_t *cls_out;     // classes after the pass
    const void *fld_c;    // C - c_ref (pitched)
    int dbl;              // fld_c stored as FP64 (else FP32)
    float c_ref;
    double c_thresh;
    uint64_t seed, cycle, lim;  // convert when (h >> 11) < lim = floor(prob * 2^53)
    unsigned long long *count;
};

}  // namespace mfc
