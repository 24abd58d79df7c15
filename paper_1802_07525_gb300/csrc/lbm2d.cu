// 2-D instantiations of the fused stream-collide kernel (flow D2Q9, transport D2Q5).
#include "mfc_internal.h"

namespace mfc {

template <typename ST, bool FLOW, bool ADE>
static cudaError_t launch_mode(const StepArgs<2, ST> &a, const StepHost &h, cudaStream_t s)
{
    switch (h.mode) {
    case MODE_PLAIN: lbm_step_kernel<2, ST, FLOW, ADE, MODE_PLAIN><<<h.grid, h.block, 0, s>>>(a); break;
    case MODE_WRITE: lbm_step_kernel<2, ST, FLOW, ADE, MODE_WRITE><<<h.grid, h.block, 0, s>>>(a); break;
    default: lbm_step_kernel<2, ST, FLOW, ADE, MODE_CHECK><<<h.grid, h.block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename ST> static cudaError_t launch_typed(const StepHost &h, cudaStream_t s)
{
    StepArgs<2, ST> a;
    a.nx = h.nx; a.ny = h.ny; a.nz = h.nz; a.px = h.px; a.plane = h.plane;
    a.bc_flow_axis = h.bc_flow_axis;
    a.rows_per_block = h.rows_per_block;
    a.fsrc = static_cast<const ST *>(h.fsrc);
    a.fdst = static_cast<ST *>(h.fdst);
    a.gsrc = static_cast<const ST *>(h.gsrc);
    a.gdst = static_cast<ST *>(h.gdst);
    a.link = static_cast<const typename Links<2>::T *>(h.link);
    a.fld_rho = h.fld_rho; a.fld_u = h.fld_u; a.fld_c = h.fld_c;
    a.partials = h.partials;
    a.omega = h.omega; a.omega_c = h.omega_c; a.k_sink = h.k_sink; a.u_scale = h.u_scale;
    a.rho_out = h.rho_out; a.c_ref = h.c_ref; a.ade_dirichlet = h.ade_dirichlet;
    for (int i = 0; i < StepArgs<2, ST>::QF; ++i) a.bb_in[i] = h.bb_in[i];
    for (int i = 0; i < StepArgs<2, ST>::QA; ++i) {
        a.gin_dev[i] = h.gin_dev[i];
        a.gout_dev[i] = h.gout_dev[i];
    }
    switch (h.kind) {
    case KIND_COUPLED: return launch_mode<ST, true, true>(a, h, s);
    case KIND_FLOW: return launch_mode<ST, true, false>(a, h, s);
    default: return launch_mode<ST, false, true>(a, h, s);
    }
}

cudaError_t launch_step_2d(const StepHost &h, cudaStream_t s)
{
    return h.half ? launch_typed<__half>(h, s) : launch_typed<float>(h, s);
}

}  // namespace mfc
