// 3-D instantiations of the fused stream-collide kernel (flow D3Q19, transport D3Q7),
// 2 nodes per thread, and of the ghost fill.
#include "mfc_internal.h"

namespace mfc {

namespace {

constexpr int VW = 2;

template <typename ST, bool FLOW, bool ADE>
cudaError_t launch_mode(const StepArgs<3, ST> &a, const StepHost &h, cudaStream_t s)
{
    switch (h.mode) {
    case MODE_PLAIN: lbm_step_kernel<3, ST, FLOW, ADE, MODE_PLAIN, VW><<<h.grid, h.block, 0, s>>>(a); break;
    case MODE_WRITE: lbm_step_kernel<3, ST, FLOW, ADE, MODE_WRITE, VW><<<h.grid, h.block, 0, s>>>(a); break;
    default: lbm_step_kernel<3, ST, FLOW, ADE, MODE_CHECK, VW><<<h.grid, h.block, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename ST> StepArgs<3, ST> make_args(const StepHost &h)
{
    StepArgs<3, ST> a;
    a.geo = h.geo;
    for (int i = 0; i < 3; ++i) a.bc[i] = h.bc[i];
    a.gpr = h.gpr;
    a.ngroups = h.ngroups;
    a.fsrc = static_cast<const ST *>(h.fsrc);
    a.fdst = static_cast<ST *>(h.fdst);
    a.gsrc = static_cast<const ST *>(h.gsrc);
    a.gdst = static_cast<ST *>(h.gdst);
    a.link = static_cast<const typename Links<3>::T *>(h.link);
    a.fld_rho = h.fld_rho; a.fld_u = h.fld_u; a.fld_c = h.fld_c;
    a.partials = h.partials;
    a.omega = h.omega; a.omega_c = h.omega_c; a.k_sink = h.k_sink; a.u_scale = h.u_scale;
    a.rho_out = h.rho_out; a.c_ref = h.c_ref; a.ade_dirichlet = h.ade_dirichlet;
    for (int i = 0; i < StepArgs<3, ST>::QF; ++i) a.bb_in[i] = h.bb_in[i];
    for (int i = 0; i < StepArgs<3, ST>::QA; ++i) {
        a.gin_dev[i] = h.gin_dev[i];
        a.gout_dev[i] = h.gout_dev[i];
    }
    return a;
}

template <typename ST> cudaError_t launch_typed(const StepHost &h, cudaStream_t s)
{
    const StepArgs<3, ST> a = make_args<ST>(h);
    switch (h.kind) {
    case KIND_COUPLED: return launch_mode<ST, true, true>(a, h, s);
    case KIND_FLOW: return launch_mode<ST, true, false>(a, h, s);
    default: return launch_mode<ST, false, true>(a, h, s);
    }
}

template <typename ST> cudaError_t fill_typed(const StepHost &h, cudaStream_t s)
{
    const StepArgs<3, ST> a = make_args<ST>(h);
    const long long N = (long long)h.geo.nx * h.geo.ny * h.geo.nz;
    const long long b = (N + 255) / 256;
    fill_ghosts_kernel<3, ST><<<(int)(b < 65535 ? b : 65535), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_3d(const StepHost &h, cudaStream_t s)
{
    return h.half ? launch_typed<__half>(h, s) : launch_typed<float>(h, s);
}

cudaError_t launch_fill_ghosts_3d(const StepHost &h, cudaStream_t s)
{
    return h.half ? fill_typed<__half>(h, s) : fill_typed<float>(h, s);
}

}  // namespace mfc
