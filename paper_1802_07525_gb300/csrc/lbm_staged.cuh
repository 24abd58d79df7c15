// TMA-staged variant of the fused 2-D stream-collide kernel (same arithmetic as
// lbm_step_kernel in lbm_kernels.cuh, bit for bit).
//
// A CTA owns a strip of W columns and sweeps a segment of rows.  For every output row t it needs,
// for each population plane i, the source row t - cy_i (the pull of Eq. 4), and for bounce-back
// (Eq. 11) the node's own opposite population, which is the source of plane opp(i) for output row
// t - cy_i.  Slot s(t) of a ring in shared memory holds, for every plane j, source row t - cy_j
// over the strip plus a halo of H elements on each side, and the link words of row t.  One thread
// issues, per slot, one bulk asynchronous copy (cp.async.bulk, the TMA engine) per plane row,
// completing on an mbarrier; the ring is filled P + 2 rows ahead of the row being computed, so the
// memory system sees deep, register-free prefetch.  Output row t reads slots t - 1, t, t + 1.
//
// Adjacent segments sweep in opposite directions, so the two CTAs that need the same halo rows
// read them at the same moment and the second read is served by L2.
//
// Waits on the mbarrier are bounded: after MFC_WAIT_LIMIT polls the CTA records an error flag,
// stops storing, keeps every thread on the same barriers, and drains the copies it issued (also
// bounded) before it returns.
#pragma once

#include "lbm_kernels.cuh"

namespace mfc {

constexpr unsigned MFC_WAIT_LIMIT = 1u << 22;

struct StagedArgs {
    int nstrips;    // strips of W columns
    int seg_rows;   // rows per segment
    int *err;       // set to 1 when a wait gives up
};

// A staged population from shared memory, as FP32.
__device__ __forceinline__ float ldsf(const float *p) { return *p; }
__device__ __forceinline__ float ldsf(const __half *p) { return __half2float(*p); }

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Poll the phase of an mbarrier; false when the poll limit is reached.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase)
{
    const unsigned a = smem_u32(bar);
    for (unsigned it = 0; it < MFC_WAIT_LIMIT; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global to shared
// memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Shared-memory footprint of one slot, and of the whole ring with its barriers.
template <typename ST, int W, bool FLOW, bool ADE>
struct StagedLayout {
    static constexpr int H = 16 / (int)sizeof(ST);  // halo elements each side (16-byte aligned copies)
    static constexpr int WC = W + 2 * H;             // elements per staged plane row
    static constexpr int NPF = FLOW ? 9 : 0;
    static constexpr int NPA = ADE ? 5 : 0;
    static constexpr int ROW_BYTES = WC * (int)sizeof(ST);
    static constexpr int LINK_BYTES = W * 2;
    static constexpr int SLOT_BYTES = ((NPF + NPA) * ROW_BYTES + LINK_BYTES + 15) / 16 * 16;
    static constexpr int bytes(int R) { return R * SLOT_BYTES + R * 8; }
};

template <typename ST, bool FLOW, bool ADE, int MODE, int W, int R>
__global__ void __launch_bounds__(W) lbm_staged_kernel(const StepArgs<2, ST> a, const StagedArgs sa)
{
    using F = FlowSet<2>;
    using A = AdeSet<2>;
    using LK = Links<2>;
    using LY = StagedLayout<ST, W, FLOW, ADE>;
    constexpr int H = LY::H;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + R * LY::SLOT_BYTES);
    const Geo &g = a.geo;
    const int tid = threadIdx.x;

    const int strip = blockIdx.x % sa.nstrips, seg = blockIdx.x / sa.nstrips;
    const int x0 = strip * W;
    const int yb = seg * sa.seg_rows;
    const int ye = min(g.ny, yb + sa.seg_rows);
    const int n = ye - yb;  // output rows of this CTA (>= 1)
    const int dir = (seg & 1) ? -1 : 1;
    const int tfirst = dir > 0 ? yb : ye - 1;
    const int nloads = n + 2;  // rows tfirst - dir ... tlast + dir

    double acc[NSUM];
#pragma unroll
    for (int m = 0; m < NSUM; ++m) acc[m] = 0.0;
    bool failed = false;

    // Issue the copies of load m (output row r = tfirst + (m - 1) * dir) into slot m % R.
    auto issue = [&](int m) {
        const int r = tfirst + (m - 1) * dir;
        unsigned char *slot = smem + (m % R) * LY::SLOT_BYTES;
        unsigned bytes = 0;
        // count first, then arm the barrier, then copy
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) mbar_expect_tx(&bars[m % R], bytes);
            int pl = 0;
            if (FLOW) {
                for (int j = 0; j < F::Q; ++j, ++pl) {
                    const int row = r - F::c(j, 1);
                    if (row < -1 || row > g.ny) continue;
                    if (pass == 0) bytes += LY::ROW_BYTES;
                    else bulk_g2s(slot + pl * LY::ROW_BYTES, a.fsrc + (long long)j * g.plane + g.at(x0 - H, row, 0),
                                  LY::ROW_BYTES, &bars[m % R]);
                }
            }
            if (ADE) {
                for (int j = 0; j < A::Q; ++j, ++pl) {
                    const int row = r - A::c(j, 1);
                    if (row < -1 || row > g.ny) continue;
                    if (pass == 0) bytes += LY::ROW_BYTES;
                    else bulk_g2s(slot + pl * LY::ROW_BYTES, a.gsrc + (long long)j * g.plane + g.at(x0 - H, row, 0),
                                  LY::ROW_BYTES, &bars[m % R]);
                }
            }
            if (r >= 0 && r < g.ny) {
                if (pass == 0) bytes += LY::LINK_BYTES;
                else bulk_g2s(slot + (LY::NPF + LY::NPA) * LY::ROW_BYTES, a.link + g.at(x0, r, 0), LY::LINK_BYTES,
                              &bars[m % R]);
            }
        }
    };

    int issued = 0;  // loads issued so far (thread 0 only)
    if (tid == 0) {
        for (int s = 0; s < R; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        for (int m = 0; m < R && m < nloads; ++m) issue(issued++);
    }
    __syncthreads();

    const int x = x0 + tid;
    const bool valid = x < g.nx;
    for (int k = 0; k < n; ++k) {
        // loads k, k+1, k+2 hold rows t - dir, t, t + dir; each slot is used for three rows
        for (int m = k; m <= k + 2; ++m)
            if (!failed && m >= k + 2 - (k == 0 ? 2 : 0))
                if (!mbar_wait(&bars[m % R], (m / R) & 1)) failed = true;
        const int t = tfirst + k * dir;
        // slot of output row tt (tt in t-1..t+1)
        auto slot_of = [&](int tt) -> const unsigned char * {
            const int m = (tt - tfirst) * dir + 1;
            return smem + (m % R) * LY::SLOT_BYTES;
        };
        const unsigned char *cur = slot_of(t);
        const uint32_t L = reinterpret_cast<const uint16_t *>(cur + (LY::NPF + LY::NPA) * LY::ROW_BYTES)[tid];
        const long long k0 = g.at(x, t, 0);
        float u[2] = {0.f, 0.f};

        if (FLOW) {
            float d[F::Q];
#pragma unroll
            for (int i = 0; i < F::Q; ++i) {
                const bool bb = i > 0 && ((L >> i) & 1u);
                if (!bb) {
                    d[i] = ldsf(reinterpret_cast<const ST *>(cur + i * LY::ROW_BYTES) + tid + H - F::c(i, 0));
                } else {
                    const unsigned char *sl = slot_of(t - F::c(i, 1));
                    d[i] = ldsf(reinterpret_cast<const ST *>(sl + F::opp(i) * LY::ROW_BYTES) + tid + H);
                }
            }
            const bool open = !(L & (1u << LK::FLOW_SELF));
            float rp = 0.f, j0 = 0.f, j1 = 0.f;
#pragma unroll
            for (int i = 0; i < F::Q; ++i) {
                if (!open) d[i] = 0.f;
                rp += d[i];
                j0 += F::c(i, 0) * d[i];
                j1 += F::c(i, 1) * d[i];
            }
            const float inv = 1.0f / (1.0f + rp);
            u[0] = j0 * inv;
            u[1] = j1 * inv;
            const float uu = u[0] * u[0] + u[1] * u[1];
            float moved = 0.f;
#pragma unroll
            for (int i = 1; i < F::Q; ++i) {
                const float cu = F::c(i, 0) * u[0] + F::c(i, 1) * u[1];
                const float feq = F::w(i) * (rp + (1.0f + rp) * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
                const float v = kept(a.fdst, d[i] + a.omega * (feq - d[i]));
                d[i] = v;
                moved += v;
                if (valid && !failed) st(a.fdst + (long long)i * g.plane + k0, v);
            }
            d[0] = rp - moved;
            if (valid && !failed) {
                st(a.fdst + k0, d[0]);
                if (open && on_open_boundary<2>(g, a.bc, x, t, 0)) {
                    float dd[F::Q], uu2[2] = {u[0], u[1]};
#pragma unroll
                    for (int i = 0; i < F::Q; ++i) dd[i] = d[i];
                    flow_ghosts<2, ST>(a, a.fdst, x, t, 0, dd, uu2);
                }
            }
            if (MODE != MODE_PLAIN && valid && !failed) {
                if (MODE == MODE_CHECK && open) {
                    const double du0 = (double)u[0] - (double)a.fld_u[k0];
                    const double du1 = (double)u[1] - (double)a.fld_u[g.plane + k0];
                    const double u2 = (double)u[0] * u[0] + (double)u[1] * u[1];
                    acc[SUM_DU2] += du0 * du0 + du1 * du1;
                    acc[SUM_U2] += u2;
                    acc[SUM_MASS] += 1.0 + (double)rp;
                    if (!isfinite(rp) || !isfinite(u2)) acc[SUM_BAD] += 1.0;
                }
                a.fld_rho[k0] = open ? rp : 0.f;
                a.fld_u[k0] = u[0];
                a.fld_u[g.plane + k0] = u[1];
            }
        }

        if (ADE) {
            if (FLOW) {
                u[0] *= a.u_scale;
                u[1] *= a.u_scale;
            } else if (!(L & (1u << LK::FLOW_SELF)) && valid) {
                u[0] = a.fld_u[k0] * a.u_scale;
                u[1] = a.fld_u[g.plane + k0] * a.u_scale;
            }
            constexpr int PA = LY::NPF;  // first transport plane in the slot
            float e[A::Q];
#pragma unroll
            for (int i = 0; i < A::Q; ++i) {
                const bool bb = i > 0 && ((L >> (LK::ADE_SELF + i)) & 1u);
                if (!bb) {
                    e[i] = ldsf(reinterpret_cast<const ST *>(cur + (PA + i) * LY::ROW_BYTES) + tid + H - A::c(i, 0));
                } else {
                    const unsigned char *sl = slot_of(t - A::c(i, 1));
                    e[i] = ldsf(reinterpret_cast<const ST *>(sl + (PA + A::opp(i)) * LY::ROW_BYTES) + tid + H);
                }
            }
            const bool open = !(L & (1u << LK::ADE_SELF));
            float cp = 0.f;
#pragma unroll
            for (int i = 0; i < A::Q; ++i) {
                if (!open) e[i] = 0.f;
                cp += e[i];
            }
            const float sink = (L & (1u << LK::SINK)) ? a.k_sink * (a.c_ref + cp) : 0.0f;
            float moved = 0.f;
#pragma unroll
            for (int i = 1; i < A::Q; ++i) {
                const float cu = A::c(i, 0) * u[0] + A::c(i, 1) * u[1];
                const float geq = A::w(i) * (cp + (a.c_ref + cp) * cu * A::inv_cs2);
                const float v = kept(a.gdst, e[i] + a.omega_c * (geq - e[i]) - A::w(i) * sink);
                e[i] = v;
                moved += v;
                if (valid && !failed) st(a.gdst + (long long)i * g.plane + k0, v);
            }
            e[0] = cp - sink - moved;
            if (valid && !failed) {
                st(a.gdst + k0, e[0]);
                if (open && on_open_boundary<2>(g, a.bc, x, t, 0)) {
                    float ee[A::Q];
#pragma unroll
                    for (int i = 0; i < A::Q; ++i) ee[i] = e[i];
                    ade_ghosts<2, ST>(a, a.gdst, x, t, 0, ee);
                }
            }
            if (MODE != MODE_PLAIN && valid && !failed) {
                if (MODE == MODE_CHECK && open) {
                    const double Cn = (double)a.c_ref + (double)cp;
                    const double dc = (double)cp - (double)a.fld_c[k0];
                    acc[SUM_DC2] += dc * dc;
                    acc[SUM_C2] += Cn * Cn;
                    acc[SUM_C] += Cn;
                    if (L & (1u << LK::SINK)) acc[SUM_CURRENT] += (double)a.k_sink * Cn;
                    if (!isfinite(cp)) acc[SUM_BAD] += 1.0;
                }
                a.fld_c[k0] = open ? cp : -a.c_ref;
            }
        }

        __syncthreads();  // everyone is done with slot k (its last reader was output row k)
        if (tid == 0 && !failed && k + R < nloads) {
            fence_proxy_async();
            issue(issued++);
        }
    }
    // Every load was waited for by the rows that use it.  After a failed wait, set the flag and
    // wait (bounded) for the most recent copy of every slot before the shared memory goes away.
    if (failed) atomicExch(sa.err, 1);
    if (tid == 0 && failed) {
        for (int m = issued > R ? issued - R : 0; m < issued; ++m) (void)mbar_wait(&bars[m % R], (m / R) & 1);
    }
    if (MODE == MODE_CHECK) block_partials(acc, a.partials);
}

}  // namespace mfc
