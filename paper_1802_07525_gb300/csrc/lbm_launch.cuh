// Launchers of the step and ghost-fill kernels for one dimension (MFC_DIM) and one storage type
// (MFC_ST), included by one translation unit per pair so that the instantiations compile in
// parallel.  Every launch variant of the step kernel is instantiated: nodes per thread in
// {1, 2, 4} (4 only in 2-D) x own-opposite load mode in {0, 1}.
#include "lbm_staged.cuh"
#include "mfc_internal.h"

#ifndef MFC_DIM
#error "MFC_DIM must be defined"
#endif

namespace mfc {

namespace {

using ST = MFC_ST;
constexpr int D = MFC_DIM;

template <bool FLOW, bool ADE, int VW, int BB>
cudaError_t launch_v(const StepArgs<D, ST> &a, const StepHost &h, cudaStream_t s)
{
    const dim3 grid((unsigned)h.grid, (unsigned)h.geo.ny, (unsigned)h.geo.nz);
    switch (h.mode) {
    case MODE_PLAIN: lbm_step_kernel<D, ST, FLOW, ADE, MODE_PLAIN, VW, BB><<<grid, h.block, 0, s>>>(a); break;
    case MODE_WRITE: lbm_step_kernel<D, ST, FLOW, ADE, MODE_WRITE, VW, BB><<<grid, h.block, 0, s>>>(a); break;
    default: lbm_step_kernel<D, ST, FLOW, ADE, MODE_CHECK, VW, BB><<<grid, h.block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <bool FLOW, bool ADE>
cudaError_t launch_mode(const StepArgs<D, ST> &a, const StepHost &h, cudaStream_t s)
{
    switch (h.vw * 2 + (h.bb ? 1 : 0)) {
    case 2: return launch_v<FLOW, ADE, 1, 0>(a, h, s);
    case 3: return launch_v<FLOW, ADE, 1, 1>(a, h, s);
    case 4: return launch_v<FLOW, ADE, 2, 0>(a, h, s);
    case 5: return launch_v<FLOW, ADE, 2, 1>(a, h, s);
#if MFC_DIM == 2
    case 8: return launch_v<FLOW, ADE, 4, 0>(a, h, s);
    case 9: return launch_v<FLOW, ADE, 4, 1>(a, h, s);
#endif
    default: return cudaErrorInvalidValue;
    }
}

StepArgs<D, ST> make_args(const StepHost &h)
{
    StepArgs<D, ST> a;
    a.geo = h.geo;
    for (int i = 0; i < 3; ++i) a.bc[i] = h.bc[i];
    a.gpr = h.gpr;
    a.fsrc = static_cast<const ST *>(h.fsrc);
    a.fdst = static_cast<ST *>(h.fdst);
    a.gsrc = static_cast<const ST *>(h.gsrc);
    a.gdst = static_cast<ST *>(h.gdst);
    a.link = static_cast<const typename Links<D>::T *>(h.link);
    a.fld_rho = h.fld_rho; a.fld_u = h.fld_u; a.fld_c = h.fld_c;
    a.partials = h.partials;
    a.omega = h.omega; a.omega_c = h.omega_c; a.k_sink = h.k_sink; a.u_scale = h.u_scale;
    a.rho_out = h.rho_out; a.c_ref = h.c_ref; a.ade_dirichlet = h.ade_dirichlet;
    for (int i = 0; i < StepArgs<D, ST>::QF; ++i) a.bb_in[i] = h.bb_in[i];
    for (int i = 0; i < StepArgs<D, ST>::QA; ++i) {
        a.gin_dev[i] = h.gin_dev[i];
        a.gout_dev[i] = h.gout_dev[i];
    }
    return a;
}

#if MFC_DIM == 2
// ---- TMA-staged kernel (2-D) ----
constexpr int RING = 5;  // slots: the three rows in use plus two rows of prefetch

template <bool FLOW, bool ADE, int MODE, int W> void *staged_fn()
{
    return reinterpret_cast<void *>(&lbm_staged_kernel<ST, FLOW, ADE, MODE, W, RING>);
}

template <bool FLOW, bool ADE, int W> int staged_smem()
{
    return StagedLayout<ST, W, FLOW, ADE>::bytes(RING);
}

// Resident CTAs per SM of the staged kernel for (kind, W); sets the shared-memory attribute of
// every mode of that kernel on first use.
int staged_ctas_per_sm(int kind, int W)
{
    static int cache[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    const int wi = W == 128 ? 0 : 1;
    if (cache[kind][wi]) return cache[kind][wi];
    void *fns[3];
    int smem = 0;
#define MFC_FNS(FL, AD, WW)                                                                         \
    fns[0] = staged_fn<FL, AD, MODE_PLAIN, WW>();                                                   \
    fns[1] = staged_fn<FL, AD, MODE_WRITE, WW>();                                                   \
    fns[2] = staged_fn<FL, AD, MODE_CHECK, WW>();                                                   \
    smem = staged_smem<FL, AD, WW>();
    if (kind == KIND_COUPLED) {
        if (W == 128) { MFC_FNS(true, true, 128) } else { MFC_FNS(true, true, 256) }
    } else if (kind == KIND_FLOW) {
        if (W == 128) { MFC_FNS(true, false, 128) } else { MFC_FNS(true, false, 256) }
    } else {
        if (W == 128) { MFC_FNS(false, true, 128) } else { MFC_FNS(false, true, 256) }
    }
#undef MFC_FNS
    for (int i = 0; i < 3; ++i)
        cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[0], W, smem);
    if (per_sm < 1) per_sm = 1;
    cache[kind][wi] = per_sm;
    return per_sm;
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

template <bool FLOW, bool ADE, int W>
cudaError_t launch_staged_w(const StepArgs<D, ST> &a, StepHost &h, cudaStream_t s)
{
    StagedArgs sa;
    int nstrips = 1, seg_rows = 1;
    MFC_PLAN_FN(h, &nstrips, &seg_rows);
    sa.nstrips = nstrips;
    sa.seg_rows = seg_rows;
    sa.err = h.err;
    const int nseg = (h.geo.ny + seg_rows - 1) / seg_rows;
    h.nblocks = nstrips * nseg;
    const int smem = staged_smem<FLOW, ADE, W>();
    switch (h.mode) {
    case MODE_PLAIN: lbm_staged_kernel<ST, FLOW, ADE, MODE_PLAIN, W, RING><<<h.nblocks, W, smem, s>>>(a, sa); break;
    case MODE_WRITE: lbm_staged_kernel<ST, FLOW, ADE, MODE_WRITE, W, RING><<<h.nblocks, W, smem, s>>>(a, sa); break;
    default: lbm_staged_kernel<ST, FLOW, ADE, MODE_CHECK, W, RING><<<h.nblocks, W, smem, s>>>(a, sa); break;
    }
    return cudaGetLastError();
}

template <bool FLOW, bool ADE>
cudaError_t launch_staged(const StepArgs<D, ST> &a, StepHost &h, cudaStream_t s)
{
    if (h.block == 128) return launch_staged_w<FLOW, ADE, 128>(a, h, s);
    return launch_staged_w<FLOW, ADE, 256>(a, h, s);
}
#endif

}  // namespace

#if MFC_DIM == 2
void MFC_PLAN_FN(const StepHost &h, int *nstrips, int *seg_rows)
{
    const int W = h.block == 128 ? 128 : 256;
    const int per_sm = staged_ctas_per_sm(h.kind, W);
    const int target = per_sm * sm_count();
    *nstrips = (h.geo.nx + W - 1) / W;
    int nseg = (target + *nstrips - 1) / *nstrips;
    if (nseg > h.geo.ny) nseg = h.geo.ny;
    if (nseg < 1) nseg = 1;
    *seg_rows = (h.geo.ny + nseg - 1) / nseg;
}
#endif

cudaError_t MFC_STEP_FN(StepHost &h, cudaStream_t s)
{
    const StepArgs<D, ST> a = make_args(h);
#if MFC_DIM == 2
    if (h.staged) {
        switch (h.kind) {
        case KIND_COUPLED: return launch_staged<true, true>(a, h, s);
        case KIND_FLOW: return launch_staged<true, false>(a, h, s);
        default: return launch_staged<false, true>(a, h, s);
        }
    }
#endif
    h.nblocks = h.grid * h.geo.ny * h.geo.nz;
    switch (h.kind) {
    case KIND_COUPLED: return launch_mode<true, true>(a, h, s);
    case KIND_FLOW: return launch_mode<true, false>(a, h, s);
    default: return launch_mode<false, true>(a, h, s);
    }
}

cudaError_t MFC_FILL_FN(const StepHost &h, cudaStream_t s)
{
    const StepArgs<D, ST> a = make_args(h);
    const long long N = (long long)h.geo.nx * h.geo.ny * h.geo.nz;
    const long long b = (N + 255) / 256;
    fill_ghosts_kernel<D, ST><<<(int)(b < 65535 ? b : 65535), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mfc
