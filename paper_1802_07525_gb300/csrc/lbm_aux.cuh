// Reduction finalize, link-mask construction, dense conversion and biofilm growth kernels
// (included by the runtime only).  All of them walk the lattice nodes in dense order
// (x fastest) and address the pitched ghost layout through Geo::at.
#pragma once

#include "lbm_kernels.cuh"

namespace mfc {

// Lattice sums in FP64, in a fixed order and in two stages spread over many SMs (a single block
// would be bound by one SM's FP64 rate).  Stage 1: block b adds partials b, b + gridDim.x, ...
// and writes one partial; stage 2: one block adds those and writes the sums and the residuals.
__global__ void __launch_bounds__(256) finalize_stage1_kernel(const double *partials, int nblocks,
                                                               double *stage1)
{
    double acc[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = 0.0;
    for (int b = blockIdx.x + gridDim.x * threadIdx.x; b < nblocks; b += gridDim.x * blockDim.x) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) acc[m] += partials[(size_t)b * NSUM + m];
    }
    block_sum_fp64(acc, stage1 + (size_t)blockIdx.x * NSUM);
}

__global__ void __launch_bounds__(256) finalize_stage2_kernel(const double *stage1, int n1, double *results)
{
    double acc[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = 0.0;
    for (int b = threadIdx.x; b < n1; b += blockDim.x) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) acc[m] += stage1[(size_t)b * NSUM + m];
    }
    __shared__ double r[NSUM];
    block_sum_fp64(acc, r);
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int m = 0; m < NSUM; ++m) results[m] = r[m];
        results[RES_FLOW] = r[SUM_U2] > 0.0 ? sqrt(r[SUM_DU2] / r[SUM_U2])
                                            : (r[SUM_DU2] > 0.0 ? INFINITY : 0.0);
        results[RES_ADE] = r[SUM_C2] > 0.0 ? sqrt(r[SUM_DC2] / r[SUM_C2])
                                           : (r[SUM_DC2] > 0.0 ? INFINITY : 0.0);
    }
}

// Fields are stored in the lattice's arithmetic type: FP64 in the FP64 instantiation, else FP32.
__device__ __forceinline__ double load_field(const void *p, int dbl, long long k)
{
    return dbl ? reinterpret_cast<const double *>(p)[k] : (double)reinterpret_cast<const float *>(p)[k];
}
__device__ __forceinline__ void store_field(void *p, int dbl, long long k, double v)
{
    if (dbl) reinterpret_cast<double *>(p)[k] = v;
    else reinterpret_cast<float *>(p)[k] = (float)v;
}

__device__ __forceinline__ void node_xyz(const Geo &g, long long q, int *x, int *y, int *z)
{
    *x = (int)(q % g.nx);
    *y = (int)((q / g.nx) % g.ny);
    *z = (int)(q / ((long long)g.nx * g.ny));
}

// Is the link that brings a population along (cx,cy,cz) to (x,y,z) blocked (Eq. 11)?  Walls win
// over the inlet and outlet; a periodic source wraps; an outlet source moves back onto the last
// layer, whose class decides; a source beyond a cut is the neighbouring slab's node, whose class
// the halo plane gives.
template <int DIM>
__device__ __forceinline__ bool mask_blocked(const MaskArgs &m, int x, int y, int z, int cx, int cy,
                                             int cz, uint8_t bit)
{
    int s[3] = {x - cx, y - cy, z - cz};
    const int n[3] = {m.geo.nx, m.geo.ny, m.geo.nz};
    constexpr int FA = DIM == 2 ? 0 : 2;
    const int side = s[FA] < 0 ? 0 : (s[FA] >= n[FA] ? 1 : -1);
    const bool across_cut = side >= 0 && m.cut[side];
    for (int ax = 0; ax < DIM; ++ax) {
        const bool out = s[ax] < 0 || s[ax] >= n[ax];
        if (ax == FA && across_cut) continue;
        if (out && !(m.bc[ax] == BC_PERIODIC || (m.bc[ax] == BC_INOUT && ax == FA))) return true;
    }
    for (int ax = 0; ax < DIM; ++ax) {
        if (s[ax] >= 0 && s[ax] < n[ax]) continue;
        if (ax == FA && across_cut) continue;
        if (m.bc[ax] == BC_PERIODIC) {
            s[ax] = s[ax] < 0 ? s[ax] + n[ax] : s[ax] - n[ax];
        } else {
            if (s[ax] < 0) return false;  // inlet ghost
            s[ax] = n[ax] - 1;            // outlet: the last layer decides
        }
    }
    if (across_cut) {
        const uint8_t *h = m.halo_cls[side];
        const long long cross = DIM == 2 ? (long long)s[1] : s[0] + (long long)m.geo.nx * s[1];
        return h && (h[cross] & bit) != 0;
    }
    return (m.cls_new[s[0] + (long long)m.geo.nx * (s[1] + (long long)m.geo.ny * s[2])] & bit) != 0;
}

// Link words from the node classes; (re)initialise populations and fields of nodes whose class
// changed (or of every node when resetting); count the open nodes.  One thread per node on a
// (row / block, ny, nz) grid, so that no index needs a division (64-bit divisions per node made
// this kernel take milliseconds on a lattice of millions of nodes).
template <int DIM, int AQ = default_aq<DIM>()> __global__ void build_links_kernel(const MaskArgs m)
{
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM, AQ>;
    using LK = Links<DIM, AQ>;
    using LinkT = typename LK::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x < m.geo.nx) {
        const long long q = x + (long long)m.geo.nx * (y + (long long)m.geo.ny * z);
        const long long k = m.geo.at(x, y, z);
        const uint8_t c = m.cls_new[q];
        uint32_t L = 0;
        if (c & CLS_FLOW) L |= 1u << LK::FLOW_SELF;
        if (c & CLS_ADE) L |= 1u << LK::ADE_SELF;
        if (c & CLS_SINK) L |= 1u << LK::SINK;
        for (int i = 1; i < F::Q; ++i)
            if (mask_blocked<DIM>(m, x, y, z, F::c(i, 0), F::c(i, 1), F::c(i, 2), CLS_FLOW)) L |= 1u << i;
        for (int i = 1; i < A::Q; ++i)
            if (mask_blocked<DIM>(m, x, y, z, A::c(i, 0), A::c(i, 1), A::c(i, 2), CLS_ADE))
                L |= 1u << (LK::ADE_SELF + i);
        reinterpret_cast<LinkT *>(m.link)[k] = (LinkT)L;

        const uint8_t o = m.reset ? (uint8_t)(CLS_FLOW | CLS_ADE) : m.cls_old[q];
        const bool f_open = !(c & CLS_FLOW), a_open = !(c & CLS_ADE);
        if (f_open && (o & CLS_FLOW)) {  // opens up (or reset): flow at rest
            for (int i = 0; i < F::Q; ++i) {
                if (m.half) reinterpret_cast<__half *>(m.fpop)[i * m.geo.plane + k] = __float2half_rn(0.f);
                else if (m.dbl) reinterpret_cast<double *>(m.fpop)[i * m.geo.plane + k] = 0.0;
                else reinterpret_cast<float *>(m.fpop)[i * m.geo.plane + k] = 0.f;
            }
        }
        if (a_open && (o & CLS_ADE)) {  // opens up (or reset): no substrate
            for (int i = 0; i < A::Q; ++i) {
                const float v = -A::w(i) * m.c_ref;
                if (m.half) reinterpret_cast<__half *>(m.gpop)[i * m.geo.plane + k] = __float2half_rn(v);
                else if (m.dbl) reinterpret_cast<double *>(m.gpop)[i * m.geo.plane + k] = -A::wd(i) * (double)m.c_ref;
                else reinterpret_cast<float *>(m.gpop)[i * m.geo.plane + k] = v;
            }
        }
        if (m.reset || !f_open) {
            store_field(m.fld_rho, m.dbl, k, 0.0);
            for (int ax = 0; ax < DIM; ++ax) store_field(m.fld_u, m.dbl, ax * m.geo.plane + k, 0.0);
        }
        if (m.reset || !a_open) store_field(m.fld_c, m.dbl, k, -(double)m.c_ref);
        // open-node counts: one atomic per warp on each of the two counters
        const unsigned act = __activemask();
        const unsigned fo = __ballot_sync(act, f_open), ao = __ballot_sync(act, a_open);
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1) {
            if (fo) atomicAdd(&m.counts[0], (unsigned long long)__popc(fo));
            if (ao) atomicAdd(&m.counts[1], (unsigned long long)__popc(ao));
        }
    }
}

// ---- fields and populations to and from dense FP64 --------------------------------------------

__device__ __forceinline__ uint32_t read_link(const void *p, int is32, long long k)
{
    return is32 ? reinterpret_cast<const uint32_t *>(p)[k] : reinterpret_cast<const uint16_t *>(p)[k];
}

__global__ void fields_to_dense_kernel(const ConvArgs a)
{
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, q, &x, &y, &z);
        const long long k = a.geo.at(x, y, z);
        const uint32_t L = read_link(a.link, a.link32, k);
        const bool fo = !(L & (1u << a.flow_self)), ao = !(L & (1u << a.ade_self));
        if (a.rho) a.rho[q] = fo ? 1.0 + load_field(a.fld_rho, a.dbl, k) : 0.0;
        if (a.u)
            for (int ax = 0; ax < a.dim; ++ax)
                a.u[ax * N + q] = fo ? load_field(a.fld_u, a.dbl, ax * a.geo.plane + k) : 0.0;
        if (a.c) {
            // C = c_ref + (C - c_ref), added in the storage's arithmetic
            const double cd = a.dbl ? (double)a.c_ref + load_field(a.fld_c, 1, k)
                                    : (double)(a.c_ref + reinterpret_cast<const float *>(a.fld_c)[k]);
            a.c[q] = ao ? cd : 0.0;
        }
    }
}

__global__ void pop_convert_kernel(const PopArgs a)
{
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(a.geo, q, &x, &y, &z);
        const long long k = a.geo.at(x, y, z);
        const bool open = a.self_bit < 0 || !(read_link(a.link, a.link32, k) & (1u << a.self_bit));
        for (int i = 0; i < a.q; ++i) {
            const long long p = i * a.geo.plane + k;
            if (a.to_dense) {
                double v = 0.0;
                if (open) {
                    const double dv = a.half  ? (double)__half2float(reinterpret_cast<const __half *>(a.pop)[p])
                                      : a.dbl ? reinterpret_cast<const double *>(a.pop)[p]
                                              : (double)reinterpret_cast<const float *>(a.pop)[p];
                    v = dv + a.w[i] * a.offset;
                }
                a.dense[i * N + q] = v;
            } else {
                const double dv = a.dense[i * N + q] - a.w[i] * a.offset;
                if (a.half) reinterpret_cast<__half *>(a.pop)[p] = __float2half_rn((float)dv);
                else if (a.dbl) reinterpret_cast<double *>(a.pop)[p] = dv;
                else reinterpret_cast<float *>(a.pop)[p] = (float)dv;
            }
        }
    }
}

// ---- biofilm growth (simplified stand-in for the agent model of Sec. 3.3) ---------------------

// splitmix64 of Steele, Lea and Flood (OOPSLA 2014), as published by Vigna.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

template <int DIM> __global__ void biofilm_grow_kernel(const GrowArgs g)
{
    using F = FlowSet<DIM>;
    const long long N = (long long)g.geo.nx * g.geo.ny * g.geo.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        const uint8_t c = g.cls[q];
        uint8_t out = c;
        if (c == 0) {
            int x, y, z;
            node_xyz(g.geo, q, &x, &y, &z);
            bool near = false;
#pragma unroll
            for (int i = 1; i < F::Q; ++i) {
                const int sx = x + F::c(i, 0), sy = y + F::c(i, 1), sz = z + F::c(i, 2);
                if (sx < 0 || sx >= g.geo.nx || sy < 0 || sy >= g.geo.ny || sz < 0 || sz >= g.geo.nz)
                    continue;
                if (g.cls[sx + (long long)g.geo.nx * (sy + (long long)g.geo.ny * sz)] & CLS_SINK) near = true;
            }
            if (near) {
                // C in the lattice's arithmetic (FP32, or FP64 in the FP64 instantiation)
                const long long k = g.geo.at(x, y, z);
                const double C = g.dbl ? (double)g.c_ref + load_field(g.fld_c, 1, k)
                                       : (double)(g.c_ref + reinterpret_cast<const float *>(g.fld_c)[k]);
                if (C > g.c_thresh) {
                    const uint64_t h = splitmix64(g.seed ^ (g.cycle << 32) ^ (uint64_t)q);
                    if ((h >> 11) < g.lim) {
                        out = CLS_FLOW | CLS_SINK;
                        atomicAdd(g.count, 1ull);
                    }
                }
            }
        }
        g.cls_out[q] = out;
    }
}

}  // namespace mfc
