// Plain coupled steps with two nodes per thread: node (x, y, z) and (x, y + 1, z), the same
// stream-collide as step_node (Eqs. 4, 5, 9-13 with the bounce-back of Eq. 11), with the
// collision of both nodes carried out by Blackwell's paired FP32 instructions (one FFMA2, FADD2 or
// FMUL2 for the two lanes).  In FP16 storage the single-node step spends its issue slots on
// arithmetic, not on HBM (the conversions and the collision per population, at half the bytes of
// FP32); pairing halves the collision's instructions and gives every thread twice the loads in
// flight.  Loads, stores, link bits and boundary work stay per node.
//
// Pairs run along y, never along the inlet/outlet axis (x in 2-D, z in 3-D), so the inlet and
// outlet tests are the same for both nodes of a pair.  Every lane rounds as an FP32 instruction
// does, but the operations are grouped differently from step_node's (the equilibrium is formed as
// w (1 + rho') t + w rho', the momentum as the sum over c = +1 less the sum over c = -1), so the
// two forms agree to FP32 rounding, not bit for bit.  Only plain steps use the pairs; check steps
// and stored-field steps stay on step_node, which reads and writes the same buffers.
#pragma once

#include "lbm_kernels.cuh"

namespace mfc {

__device__ __forceinline__ float2 p_all(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once: the product b * -1 is exact
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, p_all(-1.0f), a); }

// Sum of v[i] over the directions with c_i[ax] == s, in index order (the loops unroll, so the
// direction tests are resolved at compile time).
template <typename SET, int N>
__device__ __forceinline__ float2 p_sum_where(const float2 (&v)[N], int ax, int s)
{
    float2 r = p_all(0.0f);
    bool any = false;
#pragma unroll
    for (int i = 0; i < SET::Q; ++i) {
        if (SET::c(i, ax) != s) continue;
        r = any ? p_add(r, v[i]) : v[i];
        any = true;
    }
    return r;
}

// c_i . u with unit velocity components, as s m: m is the sum of the u[ax] with c_i[ax] = +1
// less those with -1 when both signs occur, else the sum over the one sign present, s its sign.
template <typename SET, int DIM>
__device__ __forceinline__ float2 p_cdot(int i, const float2 (&u)[3], float &s)
{
    float2 pos = p_all(0.0f), neg = p_all(0.0f);
    bool hp = false, hn = false;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        if (SET::c(i, ax) == 1) {
            pos = hp ? p_add(pos, u[ax]) : u[ax];
            hp = true;
        } else if (SET::c(i, ax) == -1) {
            neg = hn ? p_add(neg, u[ax]) : u[ax];
            hn = true;
        }
    }
    s = (hp || !hn) ? 1.0f : -1.0f;
    return (hp && hn) ? p_sub(pos, neg) : (hp ? pos : neg);
}

// Store the two lanes (lane 1 only where it exists); returns the values the stores keep.
__device__ __forceinline__ float2 p_store(float *p0, float *p1, bool has1, float2 v)
{
    *p0 = v.x;
    if (has1) *p1 = v.y;
    return v;
}
__device__ __forceinline__ float2 p_store(__half *p0, __half *p1, bool has1, float2 v)
{
    const __half2 h = __float22half2_rn(v);
    *p0 = __low2half(h);
    if (has1) *p1 = __high2half(h);
    return __half22float2(h);
}

// Which plain steps run in pairs (chosen per kernel by measurement).  They must be the ones
// whose single-node steps take the reader-side boundary form.
template <int DIM, typename ST> struct PairedStep {
    static constexpr bool value = std::is_same<ST, __half>::value;
    static_assert(!value || ReaderBoundaries<DIM, ST>::step, "paired and single-node steps share one boundary form");
};

// Resident blocks of 256 threads per SM: 3-D pairs hold 2 x 19 flow populations at once (80
// registers), 2-D pairs 2 x 9 (48).  Measured on the 256x128x128 electrode and the 4096x1024
// anode: 3-D 117.5 us at 3 blocks against 121.1 at 4 and 141.8 at 2; 2-D 58.7 us at 5 blocks
// against 62.6 at 4.
template <int DIM, typename ST> struct PairOccupancy {
    static constexpr int blocks = DIM == 3 ? 3 : 5;
};

// The link words of nodes (x, y, z) and (x, y + 1, z) (the second repeats the first where y + 1 =
// ny), and the element offset of the first.
template <int DIM, typename ST>
__device__ __forceinline__ int pair_links(const StepArgs<DIM, ST> &a, int x, int y, int z, uint32_t (&L)[2])
{
    const Geo &g = a.geo;
    const int k0 = (int)g.row0 + z * (int)g.zs + y * g.px + x;
    const int k1 = y + 1 < g.ny ? k0 + g.px : k0;
    L[0] = __ldg(a.link + MFC_IDX(k0, g.plane));
    L[1] = __ldg(a.link + MFC_IDX(k1, g.plane));
    return k0;
}

// One plain coupled step of nodes (x0 + threadIdx.x, y + l, z), l = 0, 1 (lane 1 absent where
// y + 1 = ny; x < nx), given their link words, with 32-bit element offsets and the default
// transport set.  BFORM as in step_node.
template <int DIM, typename ST, int BFORM, int SINK>
__device__ __forceinline__ void step_pair(const StepArgs<DIM, ST> &a, int x0, int y, int z, const uint32_t (&L)[2])
{
    using F = FlowSet<DIM>;
    using A = AdeSet<DIM>;
    using LK = Links<DIM>;
    static_assert(std::is_same<ArithT<ST>, float>::value, "paired FP32 arithmetic");
    static_assert(!A::quadratic, "linear transport equilibrium");
    const Geo g = a.geo;
    const int x = x0 + threadIdx.x;
    const bool has1 = y + 1 < g.ny;
    const int P = (int)g.plane;
    const int k0 = (int)g.row0 + z * (int)g.zs + y * g.px + x;
    const int k[2] = {k0, has1 ? k0 + g.px : k0};
    constexpr bool READER = BFORM != B_WRITER;
    const int y1 = has1 ? y + 1 : y;
    const bool bnd_tile = BFORM == B_WRITER ? (tile_on_open_boundary<DIM>(g, a.bc, x0, blockDim.x, y, z) ||
                                               tile_on_open_boundary<DIM>(g, a.bc, x0, blockDim.x, y1, z))
                                            : BFORM == B_BOUNDARY;
    bool ghosts[2];
#pragma unroll
    for (int l = 0; l < 2; ++l)
        ghosts[l] = bnd_tile && (l == 0 || has1) &&
                    (READER ? step_writes_ghosts<DIM>(g, a.bc, x, y + l, z) : on_open_boundary<DIM>(g, a.bc, x, y + l, z));
    constexpr int FA = flow_axis<DIM>();
    static_assert(FA != 1, "pairs along y need an inlet/outlet axis other than y");
    const int pf = FA == 0 ? x : z;
    const bool inout = READER && bnd_tile && a.bc[FA] == BC_INOUT;
    const bool at_in = inout && pf == 0 && !a.cut[0];
    const bool at_out = inout && pf == (FA == 0 ? g.nx : g.nz) - 1 && !a.cut[1];

    // ---- flow: gather (bounce-back and inlet per node), moments, BGK ----
    float2 u[3] = {p_all(0.0f), p_all(0.0f), p_all(0.0f)};
    {
        float2 d[F::Q];
#pragma unroll
        for (int i = 0; i < F::Q; ++i) {
            const int off = F::c(i, 0) + F::c(i, 1) * g.px + F::c(i, 2) * (int)g.zs;
            float v[2];
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                // bounce-back, or the moving-wall value entering across the inlet
                const bool bb = i > 0 && ((L[l] >> i) & 1u);
                const bool inj = F::c(i, FA) == 1 && at_in && !bb;
                const int o = (bb || inj) ? F::opp(i) * P : i * P - off;
                v[l] = ld(a.fsrc + MFC_IDX(k[l] + o, F::Q * P));
                if (F::c(i, FA) == 1 && inj) v[l] += a.bb_in[i];
            }
            d[i] = make_float2(v[0], v[1]);
        }
        const bool open0 = !(L[0] & (1u << LK::FLOW_SELF)), open1 = !(L[1] & (1u << LK::FLOW_SELF));
#pragma unroll
        for (int i = 0; i < F::Q; ++i)  // blocked nodes hold no populations
            d[i] = make_float2(open0 ? d[i].x : 0.0f, open1 ? d[i].y : 0.0f);
        float2 rp = d[0];
#pragma unroll
        for (int i = 1; i < F::Q; ++i) rp = p_add(rp, d[i]);
        const float2 opr = p_add(p_all(1.0f), rp);
        const float2 inv = make_float2(recip(opr.x), recip(opr.y));
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax)
            u[ax] = p_mul(p_sub(p_sum_where<F>(d, ax, 1), p_sum_where<F>(d, ax, -1)), inv);
        float2 uu = p_mul(u[0], u[0]);
#pragma unroll
        for (int ax = 1; ax < DIM; ++ax) uu = p_fma(u[ax], u[ax], uu);
        const float2 muu = p_mul(p_all(-1.5f), uu);
        const float2 om = p_all(a.omega);
        // w (1 + rho') and w rho' of the two moving weight classes (faces; diagonals or edges)
        constexpr int IE = DIM == 2 ? 5 : 7;
        const float2 wo_f = p_mul(p_all(F::w(1)), opr), wr_f = p_mul(p_all(F::w(1)), rp);
        const float2 wo_e = p_mul(p_all(F::w(IE)), opr), wr_e = p_mul(p_all(F::w(IE)), rp);
        float2 moved = p_all(0.0f);
#pragma unroll
        for (int i = 1; i < F::Q; ++i) {
            float s;
            const float2 m = p_cdot<F, DIM>(i, u, s);
            // 3 cu + 9/2 cu^2 - 3/2 u.u = m (9/2 m + 3 s) - 3/2 u.u
            const float2 t = p_fma(m, p_fma(p_all(4.5f), m, p_all(3.0f * s)), muu);
            const float2 feq = i < IE ? p_fma(wo_f, t, wr_f) : p_fma(wo_e, t, wr_e);
            const float2 v = p_fma(om, p_sub(feq, d[i]), d[i]);
            const float2 vk = p_store(a.fdst + MFC_IDX(i * P + k[0], F::Q * P),
                                      a.fdst + MFC_IDX(i * P + k[1], F::Q * P), has1, v);
            moved = i == 1 ? vk : p_add(moved, vk);
        }
        p_store(a.fdst + MFC_IDX(k[0], F::Q * P), a.fdst + MFC_IDX(k[1], F::Q * P), has1, p_sub(rp, moved));
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const bool open = l == 0 ? open0 : open1;
            if (!(ghosts[l] && open)) continue;
            const float u0 = l == 0 ? u[0].x : u[0].y, u1 = l == 0 ? u[1].x : u[1].y;
            const float u2 = l == 0 ? u[2].x : u[2].y;
            if constexpr (READER) flow_ghosts_step<DIM, ST>(a, a.fdst, x, y + l, z, k[l], u0, u1, u2);
            else flow_ghosts<DIM, ST>(a, a.fdst, x, y + l, z, k[l], L[l], u0, u1, u2);
        }
    }

    // ---- transport: gather (zero flux, inlet, outlet per node), linear equilibrium, sink ----
    {
        const float2 us = p_all(a.u_scale);
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) u[ax] = p_mul(u[ax], us);  // 0 on flow-blocked nodes
        float2 e[A::Q];
#pragma unroll
        for (int i = 0; i < A::Q; ++i) {
            const int off = A::c(i, 0) + A::c(i, 1) * g.px + A::c(i, 2) * (int)g.zs;
            float v[2];
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const bool bb = i > 0 && ((L[l] >> (LK::ADE_SELF + i)) & 1u);
                const bool in_v = A::c(i, FA) == 1 && at_in && !bb;
                const bool out_v = A::c(i, FA) == -1 && at_out && !bb;
                const int o = bb ? A::opp(i) * P : i * P - (out_v ? 0 : off);
                v[l] = ld(a.gsrc + MFC_IDX(k[l] + o, A::Q * P));
                if (A::c(i, FA) == 1 && in_v) v[l] = a.gin_dev[i];
                if (A::c(i, FA) == -1 && out_v && a.ade_dirichlet) v[l] = a.gout_dev[i];
            }
            e[i] = make_float2(v[0], v[1]);
        }
        const bool open0 = !(L[0] & (1u << LK::ADE_SELF)), open1 = !(L[1] & (1u << LK::ADE_SELF));
#pragma unroll
        for (int i = 0; i < A::Q; ++i) e[i] = make_float2(open0 ? e[i].x : 0.0f, open1 ? e[i].y : 0.0f);
        float2 cp = e[0];
#pragma unroll
        for (int i = 1; i < A::Q; ++i) cp = p_add(cp, e[i]);
        const float2 Cs = p_add(p_all(a.c_ref), cp);
        // consumption (Eq. 16's substrate factor): k C, or k C K_s / (K_s + C)
        float2 sink = p_mul(make_float2((L[0] & (1u << LK::SINK)) ? a.k_sink : 0.0f,
                                        (L[1] & (1u << LK::SINK)) ? a.k_sink : 0.0f), Cs);
        if constexpr (SINK == SINK_MONOD) {
            if (L[0] & (1u << LK::SINK)) sink.x = sink.x * a.k_half * recip(a.k_half + Cs.x);
            if (L[1] & (1u << LK::SINK)) sink.y = sink.y * a.k_half * recip(a.k_half + Cs.y);
        }
        // the moving directions share one weight: w C (1 + c_i.u / cs^2) as deviations is
        // w cp +/- (w / cs^2) C u_a
        constexpr float W = A::w(1);
        const float2 wcp = p_mul(p_all(W), cp), wsink = p_mul(p_all(W), sink);
        const float2 wc_pos = p_mul(p_all(W * A::inv_cs2), Cs), wc_neg = p_mul(p_all(-W * A::inv_cs2), Cs);
        const float2 omc = p_all(a.omega_c);
        float2 moved = p_all(0.0f);
#pragma unroll
        for (int i = 1; i < A::Q; ++i) {
            float s;
            const float2 m = p_cdot<A, DIM>(i, u, s);
            const float2 geq = p_fma(s > 0.0f ? wc_pos : wc_neg, m, wcp);
            const float2 v = p_sub(p_fma(omc, p_sub(geq, e[i]), e[i]), wsink);
            const float2 vk = p_store(a.gdst + MFC_IDX(i * P + k[0], A::Q * P),
                                      a.gdst + MFC_IDX(i * P + k[1], A::Q * P), has1, v);
            moved = i == 1 ? vk : p_add(moved, vk);
        }
        p_store(a.gdst + MFC_IDX(k[0], A::Q * P), a.gdst + MFC_IDX(k[1], A::Q * P), has1,
                p_sub(p_sub(cp, sink), moved));
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const bool open = l == 0 ? open0 : open1;
            if (!(ghosts[l] && open)) continue;
            if constexpr (READER) ade_ghosts_step<DIM, ST>(a, a.gdst, x, y + l, z, k[l]);
            else ade_ghosts<DIM, ST>(a, a.gdst, x, y + l, z, k[l], L[l]);
        }
    }
}

// Plain coupled step, two rows per thread: grid (row / block, ceil(ny / 2), nz).  Both
// dimensions take the reader-side boundary form (tiles that touch no open boundary run code with
// no boundary handling): 3-D 109.9 against 117.6 us in the writer form.  The single-node steps
// of the same storage type take it too (ReaderBoundaries), so that the forms never mix on one
// lattice.
// (A loop over several row pairs per thread, loading the next pair's link words ahead, measured
// slower at every depth tried.)
template <int DIM, typename ST, int SINK>
__global__ void __launch_bounds__(256, PairOccupancy<DIM, ST>::blocks) lbm_pair_kernel(const StepArgs<DIM, ST> a)
{
    const int x0 = blockIdx.x * blockDim.x;
    const int x = x0 + (int)threadIdx.x;
    if (x >= a.geo.nx) return;
    const int y = 2 * (int)blockIdx.y;
    // 3-D: the last plane first, as in lbm_step_kernel
    const int z = DIM == 3 ? (blockIdx.z == 0 ? (int)gridDim.z - 1 : (int)blockIdx.z - 1) : 0;
    uint32_t L[2];
    pair_links(a, x, y, z, L);
    const int y1 = y + 1 < a.geo.ny ? y + 1 : y;
    if (tile_on_open_boundary<DIM>(a.geo, a.bc, x0, blockDim.x, y, z) ||
        tile_on_open_boundary<DIM>(a.geo, a.bc, x0, blockDim.x, y1, z))
        step_pair<DIM, ST, B_BOUNDARY, SINK>(a, x0, y, z, L);
    else
        step_pair<DIM, ST, B_INTERIOR, SINK>(a, x0, y, z, L);
}

}  // namespace mfc
