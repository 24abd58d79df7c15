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
// sits at row0 + z*zs + y*px + x.  The row pitch px (a multiple of 4, >= nx + 2) keeps the left
// ghost of a row in the padding of the row before it, so every pull is a literal, in-bounds
// address and the interior needs no boundary branches.  Periodic axes, the moving-wall inlet and
// the outlet are realised by the boundary nodes writing, after their collision, the values their
// readers must see into the ghost cells of the buffer the next step reads.
//
// Threads.  One thread updates VW consecutive nodes of a row (VW = 4 in 2-D, 2 in 3-D by
// default) with 128-bit (64-bit) loads and stores; the grid is (groups of a row / block, ny, nz),
// so no index needs a division.  The populations that move along x come from the neighbouring
// lane's vector through a warp shuffle; the first or last lane of a warp, and a group at the
// start or end of a row, loads that one element itself.
//
// Precision.  Flow populations are stored as deviations from rest (f_i - w_i), transport ones
// as g_i - w_i c_ref; FP32 or FP16 storage, FP32 arithmetic.  The rest population of each lattice
// is written as the conserved total (rho - 1, or C - kC) minus the stored moving populations, so
// rounding cannot drift mass or substrate.  Check steps accumulate residual, mass, substrate and
// current sums in FP64 (warp shuffles, shared memory, one partial per block).
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

template <int DIM, typename ST> struct StepArgs {
    static constexpr int QF = FlowSet<DIM>::Q;
    static constexpr int QA = AdeSet<DIM>::Q;
    using LinkT = typename Links<DIM>::T;

    Geo geo;
    int bc[3];            // boundary kind per axis
    int gpr;              // node groups per row = ceil(nx / VW); grid = (groups / block, ny, nz)
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
    float c_ref;          // offset of the stored transport populations
    int ade_dirichlet;    // transport outlet: 0 zero-gradient, 1 Dirichlet
    float bb_in[QF];      // moving-wall inlet term 2 w_i rho_in (c_i . u_in) / cs^2
    float gin_dev[QA];    // inlet ghost: w_i c_in (1 + c_i . u_in / cs^2) - w_i c_ref
    float gout_dev[QA];   // Dirichlet outlet ghost at c_out, same form
};

template <int DIM> __host__ __device__ constexpr int flow_axis() { return DIM == 2 ? 0 : 2; }

// ---- vector loads and stores -----------------------------------------------------------------

template <int VW> __device__ __forceinline__ void ldv(const float *p, float (&v)[VW])
{
    if constexpr (VW == 1) {
        v[0] = __ldg(p);
    } else if constexpr (VW == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
}

template <int VW> __device__ __forceinline__ void ldv(const __half *p, float (&v)[VW])
{
    if constexpr (VW == 1) {
        v[0] = __half2float(__ldg(p));
    } else if constexpr (VW == 4) {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
        const unsigned t = __ldg(reinterpret_cast<const unsigned *>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t));
        v[0] = a.x; v[1] = a.y;
    }
}

template <int VW> __device__ __forceinline__ void stv(float *p, const float (&v)[VW])
{
    if constexpr (VW == 1) *p = v[0];
    else if constexpr (VW == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

template <int VW> __device__ __forceinline__ void stv(__half *p, const float (&v)[VW])
{
    if constexpr (VW == 1) {
        *p = __float2half_rn(v[0]);
    } else if constexpr (VW == 4) {
        __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        uint2 t;
        t.x = *reinterpret_cast<unsigned *>(&a);
        t.y = *reinterpret_cast<unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p) = t;
    } else {
        __half2 a = __floats2half2_rn(v[0], v[1]);
        *reinterpret_cast<__half2 *>(p) = a;
    }
}

// VW link words of a group.
template <int VW, typename LinkT>
__device__ __forceinline__ void ld_links(const LinkT *p, uint32_t (&L)[VW])
{
    if constexpr (VW == 1) {
        L[0] = __ldg(p);
    } else if constexpr (sizeof(LinkT) == 2 && VW == 4) {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
        L[0] = t.x & 0xffffu; L[1] = t.x >> 16; L[2] = t.y & 0xffffu; L[3] = t.y >> 16;
    } else if constexpr (sizeof(LinkT) == 2 && VW == 2) {
        const unsigned t = __ldg(reinterpret_cast<const unsigned *>(p));
        L[0] = t & 0xffffu; L[1] = t >> 16;
    } else if constexpr (VW == 4) {
        const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
        L[0] = t.x; L[1] = t.y; L[2] = t.z; L[3] = t.w;
    } else {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
        L[0] = t.x; L[1] = t.y;
    }
}

// Store a group: one vector store when all VW nodes are lattice nodes, else node by node (the
// tail of a row whose length is not a multiple of VW; the ghost after it must survive).
template <int VW, typename T>
__device__ __forceinline__ void st_group(T *p, const float (&v)[VW], bool full, int nvalid)
{
    if (full) {
        stv<VW>(p, v);
    } else {
#pragma unroll
        for (int j = 0; j < VW; ++j)
            if (j < nvalid) st(p + j, v[j]);
    }
}

// Gather, for direction (cx, cy, cz), the VW populations pulled from the row-shifted group at
// p_row (same x0): x-shifts come from the neighbouring lane or a scalar load at a warp/row edge.
template <int VW, typename ST>
__device__ __forceinline__ void gather(const ST *p_row, int cx, bool own_left, bool own_right,
                                       float (&src)[VW])
{
    float V[VW];
    ldv<VW>(p_row, V);
    if (cx == 0) {
#pragma unroll
        for (int j = 0; j < VW; ++j) src[j] = V[j];
    } else if (cx > 0) {
        float left = __shfl_up_sync(0xffffffffu, V[VW - 1], 1);
        if (own_left) left = ld(p_row - 1);
        src[0] = left;
#pragma unroll
        for (int j = 1; j < VW; ++j) src[j] = V[j - 1];
    } else {
        float right = __shfl_down_sync(0xffffffffu, V[0], 1);
        if (own_right) right = ld(p_row + VW);
#pragma unroll
        for (int j = 0; j < VW - 1; ++j) src[j] = V[j + 1];
        src[VW - 1] = right;
    }
}

// The node group's own populations of the opposite plane, for bounce-back along bit `bit`.
template <int VW, int BB, typename ST>
__device__ __forceinline__ void own_opposite(const ST *p, const uint32_t (&L)[VW], int bit,
                                             float (&own)[VW])
{
    if (BB == 0) {
        ldv<VW>(p, own);
    } else {
        uint32_t any = 0;
#pragma unroll
        for (int j = 0; j < VW; ++j) any |= (L[j] >> bit) & 1u;
        if (any) {
            ldv<VW>(p, own);
        } else {
#pragma unroll
            for (int j = 0; j < VW; ++j) own[j] = 0.f;
        }
    }
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
            if (lane == 0)
                partials[((size_t)blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z)) * NSUM + m] = v;
        }
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
// b (the zero shift too when include_zero), wherever an interior node pulls q along c_i.
template <int DIM, typename SET, typename ST>
__device__ __forceinline__ void ghost_images(const Geo &g, const int (&bc)[3], ST *pop, int i,
                                             int bx, int by, int bz, bool include_zero, float v)
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
    for (int ix = 0; ix < nopt[0]; ++ix)
        for (int iy = 0; iy < nopt[1]; ++iy)
            for (int iz = 0; iz < nopt[2]; ++iz) {
                if (!include_zero && ix == 0 && iy == 0 && iz == 0) continue;
                const int q0 = b[0] + opts[0][ix], q1 = b[1] + opts[1][iy], q2 = b[2] + opts[2][iz];
                if (!interior<DIM>(g, q0 + SET::c(i, 0), q1 + SET::c(i, 1), q2 + SET::c(i, 2))) continue;
                st(pop + (long long)i * g.plane + g.at(q0, q1, q2), v);
            }
}

// Flow ghost writes of node p with post-collision deviations d[i] and velocity u.
template <int DIM, typename ST>
__device__ void flow_ghosts(const StepArgs<DIM, ST> &a, ST *pop, int x, int y, int z,
                            const float *d, const float *u)
{
    using F = FlowSet<DIM>;
    constexpr int FA = flow_axis<DIM>();
    const int p[3] = {x, y, z};
    const int n[3] = {a.geo.nx, a.geo.ny, a.geo.nz};
    const bool inout = a.bc[FA] == BC_INOUT;
    const float uv[3] = {u[0], u[1], DIM == 3 ? u[2] : 0.f};
    const float uu = uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2];
#pragma unroll 1
    for (int i = 1; i < F::Q; ++i) {
        ghost_images<DIM, F, ST>(a.geo, a.bc, pop, i, x, y, z, false, d[i]);
        if (!inout) continue;
        const int cf = F::c(i, FA);
        if (p[FA] == 0 && cf == 1) {  // inlet: the node's own next-step pull along c_i
            const int q0 = x - F::c(i, 0), q1 = y - F::c(i, 1), q2 = z - F::c(i, 2);
            st(pop + (long long)i * a.geo.plane + a.geo.at(q0, q1, q2), d[F::opp(i)] + a.bb_in[i]);
        }
        if (p[FA] == n[FA] - 1 && cf == -1) {  // outlet ghost fed by this last-layer node
            const float cu = F::c(i, 0) * uv[0] + F::c(i, 1) * uv[1] + F::c(i, 2) * uv[2];
            const float v = F::w(i) * (a.rho_out - 1.0f +
                                       a.rho_out * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
            int b[3] = {x, y, z};
            b[FA] = n[FA];
            ghost_images<DIM, F, ST>(a.geo, a.bc, pop, i, b[0], b[1], b[2], true, v);
        }
    }
}

// Transport ghost writes of node p with post-collision populations e[i].
template <int DIM, typename ST>
__device__ void ade_ghosts(const StepArgs<DIM, ST> &a, ST *pop, int x, int y, int z, const float *e)
{
    using A = AdeSet<DIM>;
    constexpr int FA = flow_axis<DIM>();
    const int p[3] = {x, y, z};
    const int n[3] = {a.geo.nx, a.geo.ny, a.geo.nz};
    const bool inout = a.bc[FA] == BC_INOUT;
#pragma unroll 1
    for (int i = 1; i < A::Q; ++i) {
        ghost_images<DIM, A, ST>(a.geo, a.bc, pop, i, x, y, z, false, e[i]);
        if (!inout) continue;
        const int cf = A::c(i, FA);
        if (p[FA] == 0 && cf == 1) {
            const int q0 = x - A::c(i, 0), q1 = y - A::c(i, 1), q2 = z - A::c(i, 2);
            st(pop + (long long)i * a.geo.plane + a.geo.at(q0, q1, q2), a.gin_dev[i]);
        }
        if (p[FA] == n[FA] - 1 && cf == -1) {
            int b[3] = {x, y, z};
            b[FA] = n[FA];
            ghost_images<DIM, A, ST>(a.geo, a.bc, pop, i, b[0], b[1], b[2], true,
                                     a.ade_dirichlet ? a.gout_dev[i] : e[i]);
        }
    }
}

// ---- the step kernel -------------------------------------------------------------------------

// Launch variants (chosen per lattice, the results are identical bit for bit):
//   VW  nodes per thread (1, 2 or 4);
//   BB  0: the own opposite populations are loaded for every direction, independent of the link
//       word (no load waits on another); 1: only when a node of the group bounces back.
template <int DIM, typename ST, bool FLOW, bool ADE, int MODE, int VW, int BB>
__global__ void __launch_bounds__(256) lbm_step_kernel(const StepArgs<DIM, ST> a)
{
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM>;
    using LK = Links<DIM>;
    const Geo &g = a.geo;
    const int lane = threadIdx.x & 31;
    double acc[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = 0.0;

    {
        const int gx = blockIdx.x * blockDim.x + threadIdx.x;
        const int y = blockIdx.y, z = blockIdx.z;
        const bool live = gx < a.gpr;
        // lanes past the end of the row repeat the last group, which keeps the shuffles defined
        const int x0 = VW * (live ? gx : a.gpr - 1);
        const long long k0 = g.at(x0, y, z);
        const int nvalid = live ? min(VW, g.nx - x0) : 0;
        const bool full = nvalid == VW;
        const bool own_left = lane == 0 || x0 == 0;
        const bool own_right = lane == 31 || x0 + VW >= VW * a.gpr;
        uint32_t L[VW];
        ld_links<VW>(a.link + k0, L);
        bool ghosts = false;
#pragma unroll
        for (int j = 0; j < VW; ++j)
            ghosts = ghosts || (j < nvalid && on_open_boundary<DIM>(g, a.bc, x0 + j, y, z));
        float u[VW][3];
#pragma unroll
        for (int j = 0; j < VW; ++j) u[j][0] = u[j][1] = u[j][2] = 0.f;

        if (FLOW) {
            float d[F::Q][VW];
            ldv<VW>(a.fsrc + k0, d[0]);
#pragma unroll
            for (int i = 1; i < F::Q; ++i) {
                const long long ks = k0 - ((long long)F::c(i, 1) * g.px + (long long)F::c(i, 2) * g.zs);
                float src[VW], own[VW];
                gather<VW>(a.fsrc + (long long)i * g.plane + ks, F::c(i, 0), own_left, own_right, src);
                own_opposite<VW, BB>(a.fsrc + (long long)F::opp(i) * g.plane + k0, L, i, own);
#pragma unroll
                for (int j = 0; j < VW; ++j) d[i][j] = ((L[j] >> i) & 1u) ? own[j] : src[j];
            }
            float rp[VW], moved[VW];
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                const bool open = !(L[j] & (1u << LK::FLOW_SELF));
                float r0 = 0.f, jx[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < F::Q; ++i) {
                    if (!open) d[i][j] = 0.f;  // blocked nodes hold no populations
                    r0 += d[i][j];
#pragma unroll
                    for (int ax = 0; ax < DIM; ++ax) jx[ax] += F::c(i, ax) * d[i][j];
                }
                rp[j] = r0;
                const float inv = 1.0f / (1.0f + r0);
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) u[j][ax] = jx[ax] * inv;
                moved[j] = 0.f;
            }
            // BGK relaxation of the moving populations, then the rest one closes the mass.
#pragma unroll
            for (int i = 1; i < F::Q; ++i) {
                float v[VW];
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    float cu = 0.f, uu = 0.f;
#pragma unroll
                    for (int ax = 0; ax < DIM; ++ax) {
                        cu += F::c(i, ax) * u[j][ax];
                        uu += u[j][ax] * u[j][ax];
                    }
                    const float feq = F::w(i) * (rp[j] + (1.0f + rp[j]) * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
                    v[j] = kept(a.fdst, d[i][j] + a.omega * (feq - d[i][j]));
                    d[i][j] = v[j];
                    moved[j] += v[j];
                }
                st_group<VW>(a.fdst + (long long)i * g.plane + k0, v, full, nvalid);
            }
            {
                float v[VW];
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    v[j] = rp[j] - moved[j];
                    d[0][j] = v[j];
                }
                st_group<VW>(a.fdst + k0, v, full, nvalid);
            }
            if (ghosts) {
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    if (j >= nvalid || (L[j] & (1u << LK::FLOW_SELF))) continue;
                    if (!on_open_boundary<DIM>(g, a.bc, x0 + j, y, z)) continue;
                    float dd[F::Q];
#pragma unroll
                    for (int i = 0; i < F::Q; ++i) dd[i] = d[i][j];
                    flow_ghosts<DIM, ST>(a, a.fdst, x0 + j, y, z, dd, u[j]);
                }
            }
            if (MODE != MODE_PLAIN) {
                if (MODE == MODE_CHECK) {
#pragma unroll
                    for (int j = 0; j < VW; ++j) {
                        if (j >= nvalid || (L[j] & (1u << LK::FLOW_SELF))) continue;
                        double du2 = 0.0, u2 = 0.0;
#pragma unroll
                        for (int ax = 0; ax < DIM; ++ax) {
                            const double un = u[j][ax];
                            const double dd = un - (double)a.fld_u[ax * g.plane + k0 + j];
                            du2 += dd * dd;
                            u2 += un * un;
                        }
                        acc[SUM_DU2] += du2;
                        acc[SUM_U2] += u2;
                        acc[SUM_MASS] += 1.0 + (double)rp[j];
                        if (!isfinite(rp[j]) || !isfinite(u2)) acc[SUM_BAD] += 1.0;
                    }
                }
                float v[VW];
#pragma unroll
                for (int j = 0; j < VW; ++j) v[j] = (L[j] & (1u << LK::FLOW_SELF)) ? 0.f : rp[j];
                st_group<VW>(a.fld_rho + k0, v, full, nvalid);
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) {
#pragma unroll
                    for (int j = 0; j < VW; ++j) v[j] = u[j][ax];
                    st_group<VW>(a.fld_u + ax * g.plane + k0, v, full, nvalid);
                }
            }
        }

        if (ADE) {
            if (FLOW) {
#pragma unroll
                for (int j = 0; j < VW; ++j) {
#pragma unroll
                    for (int ax = 0; ax < DIM; ++ax) u[j][ax] *= a.u_scale;  // 0 on flow-blocked nodes
                }
            } else {
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) {
                    float v[VW];
                    ldv<VW>(a.fld_u + ax * g.plane + k0, v);
#pragma unroll
                    for (int j = 0; j < VW; ++j)
                        u[j][ax] = (L[j] & (1u << LK::FLOW_SELF)) ? 0.f : v[j] * a.u_scale;
                }
            }
            float e[A::Q][VW];
            ldv<VW>(a.gsrc + k0, e[0]);
#pragma unroll
            for (int i = 1; i < A::Q; ++i) {
                const long long ks = k0 - ((long long)A::c(i, 1) * g.px + (long long)A::c(i, 2) * g.zs);
                float src[VW], own[VW];
                gather<VW>(a.gsrc + (long long)i * g.plane + ks, A::c(i, 0), own_left, own_right, src);
                own_opposite<VW, BB>(a.gsrc + (long long)A::opp(i) * g.plane + k0, L, LK::ADE_SELF + i, own);
#pragma unroll
                for (int j = 0; j < VW; ++j) e[i][j] = ((L[j] >> (LK::ADE_SELF + i)) & 1u) ? own[j] : src[j];
            }
            float cp[VW], sink[VW], moved[VW];
#pragma unroll
            for (int j = 0; j < VW; ++j) {
                const bool open = !(L[j] & (1u << LK::ADE_SELF));
                float c0 = 0.f;
#pragma unroll
                for (int i = 0; i < A::Q; ++i) {
                    if (!open) e[i][j] = 0.f;
                    c0 += e[i][j];
                }
                cp[j] = c0;
                sink[j] = (L[j] & (1u << LK::SINK)) ? a.k_sink * (a.c_ref + c0) : 0.0f;
                moved[j] = 0.f;
            }
#pragma unroll
            for (int i = 1; i < A::Q; ++i) {
                float v[VW];
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    float cu = 0.f;
#pragma unroll
                    for (int ax = 0; ax < DIM; ++ax) cu += A::c(i, ax) * u[j][ax];
                    const float geq = A::w(i) * (cp[j] + (a.c_ref + cp[j]) * cu * A::inv_cs2);
                    v[j] = kept(a.gdst, e[i][j] + a.omega_c * (geq - e[i][j]) - A::w(i) * sink[j]);
                    e[i][j] = v[j];
                    moved[j] += v[j];
                }
                st_group<VW>(a.gdst + (long long)i * g.plane + k0, v, full, nvalid);
            }
            {
                float v[VW];
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    v[j] = cp[j] - sink[j] - moved[j];
                    e[0][j] = v[j];
                }
                st_group<VW>(a.gdst + k0, v, full, nvalid);
            }
            if (ghosts) {
#pragma unroll
                for (int j = 0; j < VW; ++j) {
                    if (j >= nvalid || (L[j] & (1u << LK::ADE_SELF))) continue;
                    if (!on_open_boundary<DIM>(g, a.bc, x0 + j, y, z)) continue;
                    float ee[A::Q];
#pragma unroll
                    for (int i = 0; i < A::Q; ++i) ee[i] = e[i][j];
                    ade_ghosts<DIM, ST>(a, a.gdst, x0 + j, y, z, ee);
                }
            }
            if (MODE != MODE_PLAIN) {
                if (MODE == MODE_CHECK) {
#pragma unroll
                    for (int j = 0; j < VW; ++j) {
                        if (j >= nvalid || (L[j] & (1u << LK::ADE_SELF))) continue;
                        const double Cn = (double)a.c_ref + (double)cp[j];
                        const double dc = (double)cp[j] - (double)a.fld_c[k0 + j];
                        acc[SUM_DC2] += dc * dc;
                        acc[SUM_C2] += Cn * Cn;
                        acc[SUM_C] += Cn;
                        if (L[j] & (1u << LK::SINK)) acc[SUM_CURRENT] += (double)a.k_sink * Cn;
                        if (!isfinite(cp[j])) acc[SUM_BAD] += 1.0;
                    }
                }
                float v[VW];
#pragma unroll
                for (int j = 0; j < VW; ++j) v[j] = (L[j] & (1u << LK::ADE_SELF)) ? -a.c_ref : cp[j];
                st_group<VW>(a.fld_c + k0, v, full, nvalid);
            }
        }
    }
    if (MODE == MODE_CHECK) block_partials(acc, a.partials);
}

// Write the ghost cells of the current buffers (a.fdst, a.gdst) from the state they hold, after
// the state was set from outside a step (geometry change, parameters, a population write).
template <int DIM, typename ST>
__global__ void fill_ghosts_kernel(const StepArgs<DIM, ST> a)
{
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM>;
    using LK = Links<DIM>;
    const Geo &g = a.geo;
    const long long N = (long long)g.nx * g.ny * g.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(q % g.nx), y = (int)((q / g.nx) % g.ny), z = (int)(q / ((long long)g.nx * g.ny));
        if (!on_open_boundary<DIM>(g, a.bc, x, y, z)) continue;
        const long long k = g.at(x, y, z);
        const uint32_t L = a.link[k];
        if (!(L & (1u << LK::FLOW_SELF))) {
            float d[F::Q], rp = 0.f, j[3] = {0.f, 0.f, 0.f};
            for (int i = 0; i < F::Q; ++i) {
                d[i] = ld(a.fdst + (long long)i * g.plane + k);
                rp += d[i];
                for (int ax = 0; ax < DIM; ++ax) j[ax] += F::c(i, ax) * d[i];
            }
            float u[3] = {0.f, 0.f, 0.f};
            for (int ax = 0; ax < DIM; ++ax) u[ax] = j[ax] / (1.0f + rp);
            flow_ghosts<DIM, ST>(a, a.fdst, x, y, z, d, u);
        }
        if (!(L & (1u << LK::ADE_SELF))) {
            float e[A::Q];
            for (int i = 0; i < A::Q; ++i) e[i] = ld(a.gdst + (long long)i * g.plane + k);
            ade_ghosts<DIM, ST>(a, a.gdst, x, y, z, e);
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
    float *fld_rho, *fld_u, *fld_c;
    float c_ref;
    unsigned long long *counts;  // [0] flow-open nodes, [1] transport-open nodes
};

struct ConvArgs {
    Geo geo;
    int dim;
    const void *link;
    int link32;          // link words are 32-bit (3-D) or 16-bit (2-D)
    int flow_self, ade_self;
    const float *fld_rho, *fld_u, *fld_c;
    float c_ref;
    double *rho, *u, *c;  // dense outputs (device staging), each may be null
};

struct PopArgs {
    Geo geo;
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
    Geo geo;
    const uint8_t *cls;   // classes before the pass
    uint8_t *cls_out;     // classes after the pass
    const float *fld_c;   // C - c_ref (pitched)
    float c_ref;
    double c_thresh;
    uint64_t seed, cycle, lim;  // convert when (h >> 11) < lim = floor(prob * 2^53)
    unsigned long long *count;
};

}  // namespace mfc
