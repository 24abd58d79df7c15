// The bio-electrochemical model of the anode (Tsompanas et al., arXiv 1802.07525, Sec. 3.2,
// Eqs. 14-21), lumped over the anode and advanced on the host once per model iteration from the
// mean substrate factor that the steady lattice solve gives.  Scalar double arithmetic: there is
// nothing data-parallel here (one mediator balance per anode), so it runs on the calling thread.
#include <math.h>
#include <string.h>

#include "../../include/mfc.h"

namespace {

constexpr double FARADAY = 96485.33212;    // C / mol (SI 2019: N_A e)
constexpr double GAS_R = 8.314462618;      // J / (mol K) (SI 2019: N_A k)
constexpr double SECONDS_PER_DAY = 86400.0;

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

bool params_ok(const mfc_electro_params *p)
{
    return finite_pos(p->m_total) && p->mediator_yield >= 0.0 && finite_pos(p->gamma) && finite_pos(p->m_electrons) &&
           p->q_max >= 0.0 && finite_pos(p->k_mox) && finite_pos(p->i0) && isfinite(p->e0) && p->r_ext >= 0.0 &&
           p->r_int >= 0.0 && finite_pos(p->r_ext + p->r_int) && p->epsilon >= 0.0 && finite_pos(p->area) &&
           finite_pos(p->temperature) && finite_pos(p->volume) && p->dt >= 0.0 && isfinite(p->dt) &&
           p->substeps >= 1;
}

}  // namespace

extern "C" MFC_API mfc_status mfc_electro_default_params(mfc_electro_params *p)
{
    if (!p) return MFC_ERR_ARG;
    memset(p, 0, sizeof *p);
    // Table 1
    p->m_total = 0.05;
    p->mediator_yield = 0.5687;
    p->gamma = 663400.0;
    p->m_electrons = 2.0;
    p->q_max = 8.48;
    p->k_mox = 0.02 * p->m_total;
    p->i0 = 0.001;
    p->e0 = 0.7;
    p->r_ext = 360.0;
    p->r_int = 360.0;
    // not given by the paper: chosen values
    p->epsilon = 0.01;
    p->area = 0.048 * 0.065;  // the electrode face, 48 x 65 mm
    p->temperature = 298.15;
    // the anode compartment, 17 x 60 x 65 mm, in litres
    p->volume = 17.0 * 60.0 * 65.0 * 1e-6;
    // one model iteration (one hour) in steps of one second: an explicit step of an hour would
    // overshoot the mediator balance, whose relaxation time is about 20 s at these values
    p->dt = 1.0;
    p->substeps = 3600;
    return MFC_OK;
}

extern "C" MFC_API mfc_status mfc_electro_update(const mfc_electro_params *p, double substrate_factor,
                                                 double c_bio, double m_ox, mfc_electro_result *out)
{
    if (!p || !out || !params_ok(p)) return MFC_ERR_ARG;
    if (!(substrate_factor >= 0.0 && substrate_factor <= 1.0) || !finite_pos(c_bio)) return MFC_ERR_ARG;
    if (!(m_ox >= 0.0 && m_ox < p->m_total)) return MFC_ERR_ARG;
    const double vt = GAS_R * p->temperature / FARADAY;  // R T / F, V
    const double biomass = p->volume * c_bio;           // V_a C^bio, mg biomass
    const double m_hi = p->m_total * (1.0 - 1e-12);     // M_red stays positive
    mfc_electro_result r;
    memset(&r, 0, sizeof r);
    double mox = m_ox;
    for (int step = 0; step < p->substeps; ++step) {
        const double mred = p->m_total - mox;
        const double qa = p->q_max * substrate_factor * mox / (mox + p->k_mox);
        const double n_conc = vt * log(p->m_total / mred);
        const double s = mred / (p->epsilon + mred);
        const double a = vt / (p->m_electrons * p->area * p->i0) * (mox / mred);  // n_act / I
        const double current = (p->e0 - n_conc) * s / (p->r_int + p->r_ext + a * s);
        r.q_a = qa;
        r.n_conc = n_conc;
        r.n_act = a * current;
        r.i_cell = current;
        r.v_cell = current * p->r_ext;
        r.v_eq21 = current * (p->r_int + p->r_ext);
        const double rate = -p->mediator_yield * qa / SECONDS_PER_DAY +
                            p->gamma * current / (p->m_electrons * FARADAY * biomass);
        mox += p->dt * rate;
        if (mox < 0.0) mox = 0.0;
        if (mox > m_hi) mox = m_hi;
    }
    r.m_ox = mox;
    r.m_red = p->m_total - mox;
    *out = r;
    return MFC_OK;
}
