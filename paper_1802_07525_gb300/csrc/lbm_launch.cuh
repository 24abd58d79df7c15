// Launchers of the step, batch-step and ghost-fill kernels for one dimension (MFC_DIM), one
// storage type (MFC_ST: float, __half, or double for the FP64 instantiation) and one transport
// velocity set (MFC_AQ, default D2Q5 / D3Q7), included
// by one translation unit per combination so that the instantiations compile in parallel.  The
// batch launchers exist for the default transport sets only (MFC_BATCH_FN defined).
#include <string.h>

#include "lbm_pair.cuh"
#include "mfc_internal.h"

#ifndef MFC_DIM
#error "MFC_DIM must be defined"
#endif

namespace mfc {

namespace {

using ST = MFC_ST;
constexpr int D = MFC_DIM;
#ifdef MFC_AQ
constexpr int AQ = MFC_AQ;
#else
constexpr int AQ = default_aq<D>();
#endif
using Args = StepArgs<D, ST, AQ>;

template <bool FLOW, bool ADE, int SINK>
cudaError_t launch_sink(const Args &a, const StepHost &h, cudaStream_t s)
{
    const dim3 grid((unsigned)h.grid, (unsigned)h.geo.ny, (unsigned)h.geo.nz);
    switch (h.mode) {
    case MODE_PLAIN:
        // the plain step, the hot loop: 32-bit element offsets where the arrays allow them, and
        // coupled steps two rows per thread where that was measured faster
        if constexpr (FLOW && ADE && AQ == default_aq<D>() && PairedStep<D, ST>::value) {
            if (h.idx32) {
                const dim3 pairs((unsigned)h.grid, (unsigned)((h.geo.ny + 1) / 2), (unsigned)h.geo.nz);
                lbm_pair_kernel<D, ST, SINK><<<pairs, h.block, 0, s>>>(a);
                break;
            }
        }
        if (h.idx32) lbm_step_kernel<D, ST, FLOW, ADE, MODE_PLAIN, AQ, SINK, true><<<grid, h.block, 0, s>>>(a);
        else lbm_step_kernel<D, ST, FLOW, ADE, MODE_PLAIN, AQ, SINK><<<grid, h.block, 0, s>>>(a);
        break;
    case MODE_WRITE: lbm_step_kernel<D, ST, FLOW, ADE, MODE_WRITE, AQ, SINK><<<grid, h.block, 0, s>>>(a); break;
    default: lbm_step_kernel<D, ST, FLOW, ADE, MODE_CHECK, AQ, SINK><<<grid, h.block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

// Steps with transport take the kernels of the lattice's consumption law; flow-only steps have
// no consumption.
template <bool FLOW, bool ADE>
cudaError_t launch_mode(const Args &a, const StepHost &h, cudaStream_t s)
{
    if constexpr (ADE) {
        if (h.k_half > 0.0) return launch_sink<FLOW, ADE, SINK_MONOD>(a, h, s);
    }
    return launch_sink<FLOW, ADE, SINK_LINEAR>(a, h, s);
}

Args make_args(const StepHost &h)
{
    Args a;
    a.geo = h.geo;
    for (int i = 0; i < 3; ++i) a.bc[i] = h.bc[i];
    a.fsrc = static_cast<const ST *>(h.fsrc);
    a.fdst = static_cast<ST *>(h.fdst);
    a.gsrc = static_cast<const ST *>(h.gsrc);
    a.gdst = static_cast<ST *>(h.gdst);
    a.link = static_cast<const typename Links<D, AQ>::T *>(h.link);
    using R = typename Args::R;
    a.fld_rho = static_cast<R *>(h.fld_rho);
    a.fld_u = static_cast<R *>(h.fld_u);
    a.fld_c = static_cast<R *>(h.fld_c);
    a.partials = h.partials;
    a.omega = (R)h.omega; a.omega_c = (R)h.omega_c; a.k_sink = (R)h.k_sink; a.u_scale = (R)h.u_scale;
    a.rho_out = (R)h.rho_out; a.c_ref = (R)h.c_ref; a.ade_dirichlet = h.ade_dirichlet;
    a.cut[0] = h.cut[0];
    a.cut[1] = h.cut[1];
    a.bounds_err = h.bounds_err;
    a.k_half = (R)h.k_half;
    for (int i = 0; i < Args::QF; ++i) a.bb_in[i] = (R)h.bb_in[i];
    for (int i = 0; i < Args::QA; ++i) {
        a.gin_dev[i] = (R)h.gin_dev[i];
        a.gout_dev[i] = (R)h.gout_dev[i];
    }
    return a;
}

}  // namespace

cudaError_t MFC_STEP_FN(StepHost &h, cudaStream_t s)
{
    const Args a = make_args(h);
    h.nblocks = h.grid * h.geo.ny * h.geo.nz;
    switch (h.kind) {
    case KIND_COUPLED: return launch_mode<true, true>(a, h, s);
    case KIND_FLOW: return launch_mode<true, false>(a, h, s);
    default: return launch_mode<false, true>(a, h, s);
    }
}

#ifdef MFC_BATCH_FN
size_t MFC_ARGS_FN(const StepHost &h, void *out)
{
    const Args a = make_args(h);
    if (out) memcpy(out, &a, sizeof a);
    return sizeof a;
}

// Coupled steps only: a batch advances flow and transport of every instance together.
cudaError_t MFC_BATCH_FN(const BatchHost &h, cudaStream_t s)
{
    BatchArgs<D, ST> b;
    b.inst = static_cast<const StepArgs<D, ST> *>(h.inst);
    b.tiles = h.tiles;
    b.ntiles = h.ntiles;
    b.partials = h.partials;
    b.parity = h.parity;
    switch (h.mode) {
    case MODE_PLAIN: lbm_batch_kernel<D, ST, true, true, MODE_PLAIN><<<h.grid, h.block, 0, s>>>(b); break;
    case MODE_WRITE: lbm_batch_kernel<D, ST, true, true, MODE_WRITE><<<h.grid, h.block, 0, s>>>(b); break;
    default: lbm_batch_kernel<D, ST, true, true, MODE_CHECK><<<h.grid, h.block, 0, s>>>(b); break;
    }
    return cudaGetLastError();
}

// Resident blocks per SM of the plain batch step at `block` threads.
int MFC_OCC_FN(int block)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lbm_batch_kernel<D, ST, true, true, MODE_PLAIN>, block, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}
#endif

cudaError_t MFC_FILL_FN(const StepHost &h, cudaStream_t s)
{
    const Args a = make_args(h);
    const long long N = (long long)h.geo.nx * h.geo.ny * h.geo.nz;
    const long long b = (N + 255) / 256;
    fill_ghosts_kernel<D, ST, AQ><<<(int)(b < 65535 ? b : 65535), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mfc
