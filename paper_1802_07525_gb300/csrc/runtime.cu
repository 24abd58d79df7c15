// Lattice objects, memory, CUDA-graph step loops and the C ABI declared in include/mfc.h.
//
// A lattice owns, on one GPU: two buffers of flow populations and two of transport populations
// (pull scheme: read one, write the other), one link word per node, the node classes, the
// FP32 fields (rho - 1, u, C - c_ref) written on check steps, per-block FP64 partial sums and
// the finalized results (mirrored into pinned host memory).  Steady solves replay a captured
// CUDA graph of K steps (K-1 plain, then one check step that compares the fields with those the
// previous check stored, stores them and reduces), then read the residuals from the pinned
// mirror.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mfc.h"
#include "lbm_aux.cuh"
#include "mfc_internal.h"
#include "runtime.h"

namespace mfc {

cudaError_t launch_links(int dim, int aq, const MaskArgs &m, cudaStream_t s)
{
    const dim3 grid((unsigned)((m.geo.nx + 255) / 256), (unsigned)m.geo.ny, (unsigned)m.geo.nz);
    if (dim == 2 && aq == 9) build_links_kernel<2, 9><<<grid, 256, 0, s>>>(m);
    else if (dim == 2) build_links_kernel<2><<<grid, 256, 0, s>>>(m);
    else build_links_kernel<3><<<grid, 256, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_grow(int dim, const GrowArgs &g, cudaStream_t s)
{
    const long long N = (long long)g.geo.nx * g.geo.ny * g.geo.nz;
    const int blocks = (int)((N + 255) / 256 < 65535 * 8 ? (N + 255) / 256 : 65535 * 8);
    if (dim == 2) biofilm_grow_kernel<2><<<blocks, 256, 0, s>>>(g);
    else biofilm_grow_kernel<3><<<blocks, 256, 0, s>>>(g);
    return cudaGetLastError();
}

// Stage-1 blocks of the lattice sums (256 threads each, about 64 partials per block).
constexpr int FINAL_STAGE1_MAX = 256;

cudaError_t launch_finalize(const double *partials, int nblocks, double *stage1, double *results,
                            cudaStream_t s)
{
    int n1 = (nblocks + 63) / 64;
    if (n1 > FINAL_STAGE1_MAX) n1 = FINAL_STAGE1_MAX;
    if (n1 < 1) n1 = 1;
    finalize_stage1_kernel<<<n1, 256, 0, s>>>(partials, nblocks, stage1);
    finalize_stage2_kernel<<<1, 256, 0, s>>>(stage1, n1, results);
    return cudaGetLastError();
}

cudaError_t launch_fields_to_dense(const ConvArgs &a, cudaStream_t s)
{
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    const int blocks = (int)((N + 255) / 256 < 65535 * 8 ? (N + 255) / 256 : 65535 * 8);
    fields_to_dense_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pop_convert(const PopArgs &a, cudaStream_t s)
{
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    const int blocks = (int)((N + 255) / 256 < 65535 * 8 ? (N + 255) / 256 : 65535 * 8);
    pop_convert_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mfc

using namespace mfc;

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace {

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

mfc_status fail(mfc_lattice *L, mfc_status s, const std::string &msg)
{
    if (L) {
        L->err = msg;
        if (s == MFC_ERR_CUDA) L->sticky = s;
    } else {
        g_create_error = msg;
    }
    return s;
}

#define CK(L, call)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(L, MFC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

// Make the lattice's device current and refuse work on a lattice with a recorded CUDA error.
mfc_status enter(mfc_lattice *L)
{
    if (!L) return MFC_ERR_ARG;
    if (L->sticky != MFC_OK) return L->sticky;
    int cur = -1;
    CK(L, cudaGetDevice(&cur));
    if (cur != L->device) CK(L, cudaSetDevice(L->device));
    return MFC_OK;
}

// Checking builds: after the lattice stream was synchronised, report an out-of-range element
// offset recorded by the step kernels (site: source line; the offset).  Other builds: nothing.
mfc_status check_bounds(mfc_lattice *L)
{
#ifdef MFC_CHECK_BOUNDS
    unsigned long long rec = 0;
    CK(L, cudaMemcpy(&rec, L->bounds_err, sizeof rec, cudaMemcpyDeviceToHost));
    if (rec) {
        L->sticky = MFC_ERR_CUDA;
        return fail(L, MFC_ERR_CUDA, "element offset out of range at kernel line " +
                                         std::to_string((rec >> 40) & 0x7FFFFF) + ", offset " +
                                         std::to_string((long long)(rec & 0xFFFFFFFFFFull)));
    }
#else
    (void)L;
#endif
    return MFC_OK;
}

mfc_status check_params(const mfc_params *p, std::string *why)
{
    auto fin = [](double v) { return isfinite(v) != 0; };
    if (!p) { *why = "params is NULL"; return MFC_ERR_ARG; }
    if (!fin(p->tau) || p->tau <= 0.5) { *why = "tau must be > 0.5"; return MFC_ERR_ARG; }
    if (!fin(p->tau_c) || p->tau_c <= 0.5) { *why = "tau_c must be > 0.5"; return MFC_ERR_ARG; }
    if (!fin(p->k_sink) || p->k_sink < 0.0 || p->k_sink >= 1.0) {
        *why = "k_sink must be in [0, 1)";
        return MFC_ERR_ARG;
    }
    if (!fin(p->u_in) || !fin(p->rho_in) || !fin(p->rho_out) || !fin(p->c_in) || !fin(p->c_out) ||
        !fin(p->u_scale) || p->rho_in <= 0.0 || p->rho_out <= 0.0) {
        *why = "inlet/outlet parameters must be finite, densities > 0";
        return MFC_ERR_ARG;
    }
    if (!fin(p->k_half) || p->k_half < 0.0) {
        *why = "k_half must be finite and >= 0";
        return MFC_ERR_ARG;
    }
    if (p->ade_outlet != MFC_OUTLET_ZERO_GRADIENT && p->ade_outlet != MFC_OUTLET_DIRICHLET) {
        *why = "ade_outlet must be MFC_OUTLET_ZERO_GRADIENT or MFC_OUTLET_DIRICHLET";
        return MFC_ERR_ARG;
    }
    return MFC_OK;
}

mfc_status check_desc(const mfc_lattice_desc *d, std::string *why)
{
    if (!d) { *why = "desc is NULL"; return MFC_ERR_ARG; }
    if (d->dim != 2 && d->dim != 3) { *why = "dim must be 2 or 3"; return MFC_ERR_ARG; }
    const int nz = d->dim == 2 ? 1 : d->nz;
    if (d->nx < 1 || d->ny < 1 || nz < 1) { *why = "sizes must be >= 1"; return MFC_ERR_ARG; }
    if ((long long)d->nx * d->ny * nz > (1ll << 31) || d->ny > 65535 || nz > 65535) {
        *why = "lattice too large (at most 2^31 nodes, ny and nz at most 65535)";
        return MFC_ERR_ARG;
    }
    const int fa = d->dim == 2 ? 0 : 2;
    for (int a = 0; a < d->dim; ++a) {
        const int b = d->bc[a];
        if (b != MFC_BC_WALL && b != MFC_BC_PERIODIC && b != MFC_BC_INOUT) {
            *why = "unknown boundary kind";
            return MFC_ERR_ARG;
        }
        if (b == MFC_BC_INOUT && a != fa) {
            *why = "MFC_BC_INOUT is only valid on the flow axis (x in 2-D, z in 3-D)";
            return MFC_ERR_ARG;
        }
    }
    if (d->precision != MFC_FP32 && d->precision != MFC_FP16_DEV && d->precision != MFC_FP64) {
        *why = "precision must be MFC_FP32, MFC_FP16_DEV or MFC_FP64";
        return MFC_ERR_ARG;
    }
    if (!(d->ade_q == 0 || (d->dim == 2 && (d->ade_q == 5 || d->ade_q == 9)) || (d->dim == 3 && d->ade_q == 7))) {
        *why = "ade_q must be 0 (default), 5 or 9 in 2-D, 7 in 3-D";
        return MFC_ERR_ARG;
    }
    for (int s = 0; s < 2; ++s)
        if (d->cut[s] != 0 && d->cut[s] != 1) {
            *why = "cut[] must be 0 or 1";
            return MFC_ERR_ARG;
        }
    if ((d->cut[0] || d->cut[1]) && d->bc[fa] == MFC_BC_PERIODIC) {
        *why = "a lattice with a cut may not be periodic along the flow axis";
        return MFC_ERR_ARG;
    }
    return MFC_OK;
}

struct Layout {
    int dim, qf, qa;
    Geo geo;
    long long N;
    size_t st, link_bytes;
    size_t fb;  // bytes per field value: 4, or 8 in the FP64 instantiation
};

// Ghost-layer layout: row pitch px = nx + 2 rounded up to 4 (left ghost of a row in the padding
// of the row before), ghost rows y = -1 and y = ny, ghost slabs z = -1 and z = nz in 3-D, and four
// elements in front so that node (-1, -1, -1) exists; planes rounded to 64 elements (256 B).
Layout layout_of(const mfc_lattice_desc *d)
{
    Layout l;
    l.dim = d->dim;
    l.qf = d->dim == 2 ? 9 : 19;
    l.qa = d->dim == 2 ? (d->ade_q == 9 ? 9 : 5) : 7;
    Geo &g = l.geo;
    g.nx = d->nx;
    g.ny = d->ny;
    g.nz = d->dim == 2 ? 1 : d->nz;
    // pitch and front offset are multiples of 8 elements (32-byte aligned FP32 rows)
    g.px = (int)round_up((size_t)g.nx + 2, 8);
    g.zs = (long long)(g.ny + 2) * g.px;
    const int gz = d->dim == 3 ? 1 : 0;
    g.row0 = 8 + ((long long)gz * (g.ny + 2) + 1) * g.px;
    const long long last = g.at(0, g.ny + 1, g.nz - 1 + gz);  // first element past the last ghost row
    g.plane = (long long)round_up((size_t)(last + 2 * g.px + 64), 64);
    l.N = (long long)g.nx * g.ny * g.nz;
    l.st = d->precision == MFC_FP16_DEV ? 2 : (d->precision == MFC_FP64 ? 8 : 4);
    l.fb = d->precision == MFC_FP64 ? 8 : 4;
    l.link_bytes = (d->dim == 2 && l.qa == 5) ? 2 : 4;  // 9 + 9 + 1 link bits need 32-bit words
    return l;
}

// Launch shape: one thread per node, grid (row / block, ny, nz).
void choose_launch(mfc_lattice *L)
{
    L->grid = (L->nx + L->block - 1) / L->block;
    L->nblocks = L->grid * L->ny * L->nz;
}

// Blocks of the largest launch (128 threads per block): the size of the partial-sum buffer.
int max_launch_blocks(const Layout &l)
{
    return (l.geo.nx + 127) / 128 * l.geo.ny * l.geo.nz;
}

}  // namespace

long long mfc::lattice_max_elements(const mfc_lattice_desc *d)
{
    const Layout l = layout_of(d);
    return (long long)(l.qf > l.qa ? l.qf : l.qa) * l.geo.plane;
}

void mfc::fill_step(const mfc_lattice *L, int kind, int mode, StepHost *h)
{
    memset(h, 0, sizeof *h);
    h->dim = L->dim;
    h->half = L->half;
    h->dbl = L->dbl;
    h->kind = kind;
    h->mode = mode;
    h->geo = L->geo;
    for (int a = 0; a < 3; ++a) h->bc[a] = a < L->dim ? L->desc.bc[a] : MFC_BC_PERIODIC;

    h->grid = L->grid;
    h->block = L->block;
    // the largest element offset a step forms is below max(Q_flow, Q_transport) planes
    const long long qmax = L->qf > L->qa ? L->qf : L->qa;
    h->idx32 = L->offsets32 && qmax * L->geo.plane < (1ll << 31) ? 1 : 0;
    h->fsrc = L->f[L->fcur];
    h->fdst = L->f[1 - L->fcur];
    h->gsrc = L->g[L->gcur];
    h->gdst = L->g[1 - L->gcur];
    h->link = L->link;
    h->fld_rho = L->fld_rho; h->fld_u = L->fld_u; h->fld_c = L->fld_c;
    h->partials = L->partials;
    const mfc_params &p = L->prm;
    // Parameters are kept in double here and rounded once to the arithmetic type when the
    // argument block is built; the weights are that type's (FP32 constants, or FP64 ones).
    const bool dbl = L->dbl;
    h->omega = 1.0 / p.tau;
    h->omega_c = 1.0 / p.tau_c;
    h->k_sink = p.k_sink;
    h->k_half = p.k_half;
    h->u_scale = p.u_scale;
    h->rho_out = p.rho_out;
    h->c_ref = L->c_ref;
    h->ade_dirichlet = p.ade_outlet == MFC_OUTLET_DIRICHLET;
    h->cut[0] = L->desc.cut[0];
    h->cut[1] = L->desc.cut[1];
    h->bounds_err = L->bounds_err;
    const int fa = L->dim == 2 ? 0 : 2;
    for (int i = 0; i < L->qf; ++i) {
        const int ci = L->dim == 2 ? FlowSet<2>::c(i, fa) : FlowSet<3>::c(i, fa);
        const double w = L->dim == 2 ? (dbl ? FlowSet<2>::wd(i) : FlowSet<2>::w(i))
                                     : (dbl ? FlowSet<3>::wd(i) : FlowSet<3>::w(i));
        h->bb_in[i] = 2.0 * w * p.rho_in * ci * p.u_in * 3.0;
    }
    // transport inlet (and Dirichlet outlet) equilibria at the inlet velocity: linear on D2Q5 /
    // D3Q7, the quadratic form of Eq. 5 on D2Q9
    const double inv_cs2 = L->dim == 2 ? 3.0 : 4.0;
    for (int i = 0; i < L->qa; ++i) {
        int ci;
        double w, shape;
        if (L->qa == 9) {
            ci = AdeSet<2, 9>::c(i, fa);
            w = dbl ? AdeSet<2, 9>::wd(i) : AdeSet<2, 9>::w(i);
            const double cu = ci * p.u_in;
            shape = 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * p.u_in * p.u_in;
        } else {
            ci = L->dim == 2 ? AdeSet<2>::c(i, fa) : AdeSet<3>::c(i, fa);
            w = L->dim == 2 ? (dbl ? AdeSet<2>::wd(i) : AdeSet<2>::w(i)) : (dbl ? AdeSet<3>::wd(i) : AdeSet<3>::w(i));
            shape = 1.0 + ci * p.u_in * inv_cs2;
        }
        h->gin_dev[i] = w * p.c_in * shape - w * L->c_ref;
        h->gout_dev[i] = w * p.c_out * shape - w * L->c_ref;
    }
    h->aq = L->qa;
}

namespace {

// Queue one step of `kind` and swap the buffers it wrote; *nblocks receives the blocks (and
// reduction partials) of the launch.
mfc_status enqueue_step(mfc_lattice *L, int kind, int mode, int *nblocks = nullptr)
{
    StepHost h;
    fill_step(L, kind, mode, &h);
    cudaError_t e = launch_step(h, L->stream);
    if (e != cudaSuccess) return fail(L, MFC_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    if (nblocks) *nblocks = h.nblocks;
    if (kind != KIND_ADE) L->fcur ^= 1;
    if (kind != KIND_FLOW) L->gcur ^= 1;
    return MFC_OK;
}

// Rewrite the ghost cells of the current buffers from the state they hold.
mfc_status fill_ghosts(mfc_lattice *L)
{
    StepHost h;
    fill_step(L, KIND_COUPLED, MODE_PLAIN, &h);
    h.fsrc = h.fdst = L->f[L->fcur];
    h.gsrc = h.gdst = L->g[L->gcur];
    cudaError_t e = launch_fill_ghosts(h, L->stream);
    if (e != cudaSuccess) return fail(L, MFC_ERR_CUDA, std::string("ghost fill: ") + cudaGetErrorString(e));
    return MFC_OK;
}

// Queue n >= 1 steps ending with a residual check (which compares the fields with those stored
// by the last step before the block, and stores its own) or with a plain field store.
mfc_status enqueue_block(mfc_lattice *L, int kind, int n, bool check)
{
    int nb = L->nblocks;
    for (int s = 0; s < n; ++s) {
        int mode = MODE_PLAIN;
        if (s == n - 1) mode = check ? MODE_CHECK : MODE_WRITE;
        mfc_status st = enqueue_step(L, kind, mode, &nb);
        if (st != MFC_OK) return st;
    }
    if (check) {
        CK(L, launch_finalize(L->partials, nb, L->partials + (size_t)L->max_blocks * NSUM, L->results_d,
                              L->stream));
        CK(L, cudaMemcpyAsync(L->results_h, L->results_d, sizeof(double) * NRESULT,
                              cudaMemcpyDeviceToHost, L->stream));
    }
    return MFC_OK;
}

void drop_graphs(mfc_lattice *L)
{
    for (auto &g : L->graphs) cudaGraphExecDestroy(g.exec);
    L->graphs.clear();
}

// The graph of K steps ending with a check, for the current buffer parity.
mfc_status graph_for(mfc_lattice *L, int kind, int K, cudaGraphExec_t *out)
{
    for (auto &g : L->graphs)
        if (g.kind == kind && g.K == K && g.fpar == L->fcur && g.gpar == L->gcur) {
            *out = g.exec;
            return MFC_OK;
        }
    const int f0 = L->fcur, g0 = L->gcur;
    CK(L, cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
    mfc_status st = enqueue_block(L, kind, K, true);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(L->stream, &graph);
    L->fcur = f0;  // capture recorded the launches; nothing ran
    L->gcur = g0;
    if (st != MFC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return fail(L, MFC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(L, MFC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    L->graphs.push_back({kind, K, f0, g0, exec});
    *out = exec;
    return MFC_OK;
}

// Wait for the queued work; with a deadline, poll an event and give up at the deadline.
mfc_status wait_done(mfc_lattice *L, double deadline_s, bool *timed_out)
{
    *timed_out = false;
    CK(L, cudaEventRecord(L->done, L->stream));
    if (deadline_s <= 0.0) {
        CK(L, cudaEventSynchronize(L->done));
        return MFC_OK;
    }
    using clk = std::chrono::steady_clock;
    for (;;) {
        cudaError_t e = cudaEventQuery(L->done);
        if (e == cudaSuccess) return MFC_OK;
        if (e != cudaErrorNotReady) return fail(L, MFC_ERR_CUDA, std::string("event: ") + cudaGetErrorString(e));
        const double now = std::chrono::duration<double>(clk::now().time_since_epoch()).count();
        if (now > deadline_s) {
            *timed_out = true;
            CK(L, cudaEventSynchronize(L->done));  // the queued work is bounded: let it finish
            return MFC_OK;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

double mfc::now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {

// Run one solver (or both, concurrently) to steady state.  Steps run in blocks of K ending with a
// check; the residual of a check is the mean relative change per step since the previous one,
// ||v^n - v^m|| / ((n - m) ||v^n||), where the fields of step m were stored by the previous
// check, or, for the first block, by the last step run before the call.
mfc_status run_phase(mfc_lattice *L, int kind, double tol_flow, double tol_ade, long max_steps, int K,
                     double deadline, long *steps, double *res_f, double *res_a, bool *converged)
{
    *steps = 0;
    *converged = false;
    while (*steps < max_steps) {
        const long left = max_steps - *steps;
        const int n = left >= K ? K : (int)left;
        mfc_status st;
        if (n == K) {
            cudaGraphExec_t exec;
            st = graph_for(L, kind, K, &exec);
            if (st != MFC_OK) return st;
            CK(L, cudaGraphLaunch(exec, L->stream));
            if (kind != KIND_ADE && (K & 1)) L->fcur ^= 1;
            if (kind != KIND_FLOW && (K & 1)) L->gcur ^= 1;
        } else {
            st = enqueue_block(L, kind, n, true);
            if (st != MFC_OK) return st;
        }
        bool to = false;
        st = wait_done(L, deadline, &to);
        if (st != MFC_OK) return st;
        *steps += n;
        const double *r = L->results_h;
        const double rf = r[RES_FLOW] / n, ra = r[RES_ADE] / n;
        if (kind != KIND_ADE) *res_f = rf;
        if (kind != KIND_FLOW) {
            *res_a = ra;
            L->last_current = r[SUM_CURRENT];
        }
        if (r[SUM_BAD] > 0.0 || !isfinite(r[SUM_MASS]) || !isfinite(r[SUM_C]) || isnan(rf) || isnan(ra))
            return MFC_ERR_NONFINITE;
        if (r[SUM_FAST] > 0.0) return MFC_ERR_UNSTABLE;
        const bool okf = kind == KIND_ADE || rf < tol_flow;
        const bool oka = kind == KIND_FLOW || ra < tol_ade;
        if (okf && oka) {
            *converged = true;
            return MFC_OK;
        }
        if (to) return MFC_ERR_TIMEOUT;
    }
    return MFC_OK;
}

// Device allocation of a lattice buffer, zero-filled (ghosts and padding start defined): from
// the lattice's pool on its stream, or with cudaMalloc.
#ifdef MFC_CHECK_BOUNDS
// Checking builds: every buffer sits between two guard regions of a known byte pattern, which
// mfc_check_canaries compares after the fact.
constexpr size_t GUARD = 256;
constexpr unsigned char GUARD_BYTE = 0xA5;
#else
constexpr size_t GUARD = 0;
#endif

bool dev_alloc(mfc_lattice *L, void **p, size_t bytes)
{
    *p = nullptr;
    const size_t body = GUARD ? round_up(bytes, GUARD) : bytes;
    const size_t total = body + 2 * GUARD;
    void *base = nullptr;
    if (L->pool) {
        if (cudaMallocFromPoolAsync(&base, total, L->pool, L->stream) != cudaSuccess ||
            cudaMemsetAsync(base, 0, total, L->stream) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    } else {
        if (cudaMalloc(&base, total) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (cudaMemset(base, 0, total) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
#ifdef MFC_CHECK_BOUNDS
    // the guards go on after the zero fill: that ran on the legacy stream (no pool) or on the
    // lattice stream (pool), so order the lattice stream behind the legacy one first
    char *b = static_cast<char *>(base);
    if (!L->pool) cudaDeviceSynchronize();
    cudaMemsetAsync(b, GUARD_BYTE, GUARD, L->stream);
    cudaMemsetAsync(b + GUARD + body, GUARD_BYTE, GUARD, L->stream);
    if (!L->pool) cudaStreamSynchronize(L->stream);
    L->guards.push_back({b, body});
#endif
    *p = static_cast<char *>(base) + GUARD;
    return true;
}

void dev_free(mfc_lattice *L, void *p)
{
    if (!p) return;
    char *base = static_cast<char *>(p) - GUARD;
#ifdef MFC_CHECK_BOUNDS
    for (size_t i = 0; i < L->guards.size(); ++i)
        if (L->guards[i].first == base) {
            L->guards.erase(L->guards.begin() + (long)i);
            break;
        }
#endif
    if (L->pool) cudaFreeAsync(base, L->stream);
    else cudaFree(base);
}

void release(mfc_lattice *L)
{
    if (!L) return;
    drop_graphs(L);
    for (int b = 0; b < 2; ++b) {
        dev_free(L, L->f[b]);
        dev_free(L, L->g[b]);
    }
    dev_free(L, L->link);
    dev_free(L, L->cls_cur);
    dev_free(L, L->cls_tmp);
    dev_free(L, L->fld_rho);
    dev_free(L, L->fld_u);
    dev_free(L, L->fld_c);
    dev_free(L, L->partials);
    dev_free(L, L->results_d);
    dev_free(L, L->counts_d);
    dev_free(L, L->staging);
    dev_free(L, L->bounds_err);
    dev_free(L, L->biomass);
    dev_free(L, L->halo_cls[0]);
    dev_free(L, L->halo_cls[1]);
    dev_free(L, L->agent_keys);
    dev_free(L, L->agent_list);
    dev_free(L, L->agent_mark);
    dev_free(L, L->agent_path);
    dev_free(L, L->agent_state);
    if (L->results_h) cudaFreeHost(L->results_h);
    if (L->counts_h) cudaFreeHost(L->counts_h);
    if (L->done) cudaEventDestroy(L->done);
    if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
}

mfc_status ensure_staging(mfc_lattice *L, size_t bytes)
{
    if (L->staging_bytes >= bytes) return MFC_OK;
    dev_free(L, L->staging);
    L->staging = nullptr;
    L->staging_bytes = 0;
    void *p = nullptr;
    if (!dev_alloc(L, &p, bytes)) return fail(L, MFC_ERR_OOM, "staging allocation failed");
    L->staging = static_cast<double *>(p);
    L->staging_bytes = bytes;
    return MFC_OK;
}

mfc_status apply_geometry(mfc_lattice *L, const uint8_t *dev_cls_new, int reset)
{
    MaskArgs m;
    memset(&m, 0, sizeof m);
    m.geo = L->geo;
    for (int a = 0; a < 3; ++a) m.bc[a] = a < L->dim ? L->desc.bc[a] : MFC_BC_PERIODIC;
    m.cls_new = dev_cls_new;
    m.cls_old = L->cls_cur;
    m.reset = reset;
    m.link = L->link;
    m.fpop = L->f[L->fcur];
    m.gpop = L->g[L->gcur];
    m.half = L->half;
    m.dbl = L->dbl;
    m.fld_rho = L->fld_rho; m.fld_u = L->fld_u; m.fld_c = L->fld_c;
    m.c_ref = L->c_ref;
    m.counts = L->counts_d;
    for (int s = 0; s < 2; ++s) {
        m.cut[s] = L->desc.cut[s];
        m.halo_cls[s] = L->halo_cls[s];
    }
    CK(L, cudaMemsetAsync(L->counts_d, 0, 2 * sizeof(unsigned long long), L->stream));
    CK(L, launch_links(L->dim, L->qa, m, L->stream));
    mfc_status st = fill_ghosts(L);
    if (st != MFC_OK) return st;
    CK(L, cudaMemcpyAsync(L->counts_h, L->counts_d, 2 * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, L->stream));
    CK(L, cudaStreamSynchronize(L->stream));
    L->flow_open = (long)L->counts_h[0];
    L->ade_open = (long)L->counts_h[1];
    if (dev_cls_new != L->cls_cur) {
        uint8_t *t = L->cls_cur;
        L->cls_cur = L->cls_tmp;
        L->cls_tmp = t;
    }
    return MFC_OK;
}

}  // namespace

// Lattice services for the other translation units of the library (the agent-based biofilm).
mfc_status mfc::lattice_enter(mfc_lattice *L) { return enter(L); }
mfc_status mfc::lattice_fail(mfc_lattice *L, mfc_status s, const std::string &msg) { return fail(L, s, msg); }
bool mfc::lattice_alloc(mfc_lattice *L, void **p, size_t bytes) { return dev_alloc(L, p, bytes); }
void mfc::lattice_free(mfc_lattice *L, void *p) { dev_free(L, p); }
mfc_status mfc::lattice_apply_classes(mfc_lattice *L, const uint8_t *dev_cls, int reset)
{
    return apply_geometry(L, dev_cls, reset);
}

// The fields as dense doubles, queued on the lattice stream into host buffers (each may be null).
mfc_status mfc::lattice_fields_async(mfc_lattice *L, double *rho, double *u, double *c)
{
    mfc_status st = MFC_OK;
    const size_t N = (size_t)L->N;
    st = ensure_staging(L, (size_t)(2 + L->dim) * N * sizeof(double));
    if (st != MFC_OK) return st;
    ConvArgs a;
    memset(&a, 0, sizeof a);
    a.geo = L->geo;
    a.dim = L->dim;
    a.link = L->link;
    a.link32 = L->link32;
    a.flow_self = 0;
    a.ade_self = L->qf;
    a.dbl = L->dbl;
    a.fld_rho = L->fld_rho; a.fld_u = L->fld_u; a.fld_c = L->fld_c;
    a.c_ref = L->c_ref;
    a.rho = rho ? L->staging : nullptr;
    a.u = u ? L->staging + N : nullptr;
    a.c = c ? L->staging + (1 + L->dim) * N : nullptr;
    if (rho || u || c) {
        CK(L, launch_fields_to_dense(a, L->stream));
        if (rho) CK(L, cudaMemcpyAsync(rho, a.rho, N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        if (u) CK(L, cudaMemcpyAsync(u, a.u, L->dim * N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        if (c) CK(L, cudaMemcpyAsync(c, a.c, N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    }
    return MFC_OK;
}

// Free a lattice whose device buffers come from a stream-ordered pool without waiting for its
// stream: the frees are queued behind the work already on it.
void mfc::lattice_destroy_ordered(mfc_lattice *L)
{
    if (!L) return;
    release(L);
    delete L;
}

mfc_status mfc::lattice_create(const mfc_lattice_desc *desc, const mfc_params *params, cudaMemPool_t pool,
                               mfc_lattice **out, std::string *why_out)
{
    std::string &why = *why_out;
    if (!out) { why = "out is NULL"; return MFC_ERR_ARG; }
    *out = nullptr;
    mfc_status st = check_desc(desc, &why);
    if (st == MFC_OK) st = check_params(params, &why);
    if (st != MFC_OK) return st;
    if (pool && !desc->stream) { why = "a pooled lattice needs a stream"; return MFC_ERR_ARG; }

    int ndev = 0;
    cudaError_t de = cudaGetDeviceCount(&ndev);
    if (de != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        why = std::string("no CUDA device: ") + cudaGetErrorString(de);
        return MFC_ERR_CUDA;
    }
    mfc_lattice *L = new (std::nothrow) mfc_lattice();
    if (!L) { why = "host allocation failed"; return MFC_ERR_OOM; }
    L->pool = pool;
    L->desc = *desc;
    if (desc->dim == 2) {
        L->desc.nz = 1;
        L->desc.bc[2] = MFC_BC_PERIODIC;
    }
    L->prm = *params;
    Layout l = layout_of(desc);
    L->dim = l.dim; L->qf = l.qf; L->qa = l.qa;
    L->geo = l.geo;
    L->nx = l.geo.nx; L->ny = l.geo.ny; L->nz = l.geo.nz;
    L->N = l.N;
    L->st_bytes = l.st;
    L->half = desc->precision == MFC_FP16_DEV;
    L->dbl = desc->precision == MFC_FP64;
    L->link32 = l.link_bytes == 4;
    // transport storage offset: 0, so that the no-substrate start state is stored exactly
    L->c_ref = 0.0f;
    cudaGetDevice(&L->device);
    L->block = DEFAULT_BLOCK;
    L->max_blocks = max_launch_blocks(l);
    choose_launch(L);

    // the stream first: pooled buffers are allocated on it
    cudaError_t e = cudaSuccess;
    if (desc->stream) {
        L->stream = (cudaStream_t)desc->stream;
    } else {
        e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            L->stream = nullptr;
            why = std::string("create: ") + cudaGetErrorString(e);
            delete L;
            return MFC_ERR_CUDA;
        }
        L->own_stream = true;
    }
    auto dalloc = [&](void **p, size_t bytes) -> bool {
        if (!dev_alloc(L, p, bytes)) return false;
        L->bytes += bytes;
        return true;
    };
    const long long P = l.geo.plane;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        ok = ok && dalloc(&L->f[b], (size_t)l.qf * P * l.st);
        ok = ok && dalloc(&L->g[b], (size_t)l.qa * P * l.st);
    }
    ok = ok && dalloc(&L->link, (size_t)P * l.link_bytes);
    ok = ok && dalloc((void **)&L->cls_cur, round_up((size_t)l.N, 256));
    ok = ok && dalloc((void **)&L->cls_tmp, round_up((size_t)l.N, 256));
    ok = ok && dalloc(&L->fld_rho, (size_t)P * l.fb);
    ok = ok && dalloc(&L->fld_u, (size_t)l.dim * P * l.fb);
    ok = ok && dalloc(&L->fld_c, (size_t)P * l.fb);
    // per-block partials, then the stage-1 sums of the finalize
    ok = ok && dalloc((void **)&L->partials, ((size_t)L->max_blocks + FINAL_STAGE1_MAX) * NSUM * sizeof(double));
    ok = ok && dalloc((void **)&L->results_d, NRESULT * sizeof(double));
    ok = ok && dalloc((void **)&L->counts_d, 2 * sizeof(unsigned long long));
#ifdef MFC_CHECK_BOUNDS
    ok = ok && dalloc((void **)&L->bounds_err, sizeof(unsigned long long));
#endif
    if (!ok) {
        release(L);
        delete L;
        why = "device allocation failed";
        return MFC_ERR_OOM;
    }
    e = cudaHostAlloc((void **)&L->results_h, NRESULT * sizeof(double), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&L->counts_h, 2 * sizeof(unsigned long long), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        why = std::string("create: ") + cudaGetErrorString(e);
        release(L);
        delete L;
        return MFC_ERR_CUDA;
    }
    memset(L->results_h, 0, NRESULT * sizeof(double));
    // every node open, rest state
    e = cudaMemsetAsync(L->cls_cur, 0, round_up((size_t)l.N, 256), L->stream);
    if (e != cudaSuccess) {
        why = std::string("create: ") + cudaGetErrorString(e);
        release(L);
        delete L;
        return MFC_ERR_CUDA;
    }
    st = apply_geometry(L, L->cls_cur, 1);
    if (st != MFC_OK) {
        why = L->err;
        release(L);
        delete L;
        return st;
    }
    *out = L;
    return MFC_OK;
}

mfc_status mfc::validate_lattice(const mfc_lattice_desc *desc, const mfc_params *params, std::string *why)
{
    mfc_status st = check_desc(desc, why);
    if (st == MFC_OK) st = check_params(params, why);
    return st;
}

extern "C" {

MFC_API size_t mfc_lattice_bytes(const mfc_lattice_desc *desc)
{
    std::string why;
    if (check_desc(desc, &why) != MFC_OK) return 0;
    Layout l = layout_of(desc);
    size_t b = 0;
    const long long P = l.geo.plane;
    b += 2 * (size_t)l.qf * P * l.st;             // flow A/B
    b += 2 * (size_t)l.qa * P * l.st;             // transport A/B
    b += (size_t)P * l.link_bytes;                // links
    b += 2 * round_up((size_t)l.N, 256);          // classes (current, next)
    b += (size_t)(2 + l.dim) * P * l.fb;          // fields
    b += ((size_t)max_launch_blocks(l) + FINAL_STAGE1_MAX) * NSUM * sizeof(double);  // partials
    b += 4096;
    return b;
}

MFC_API mfc_status mfc_create_lattice(const mfc_lattice_desc *desc, const mfc_params *params,
                                      mfc_lattice **out)
{
    std::string why;
    mfc_status st = lattice_create(desc, params, nullptr, out, &why);
    if (st != MFC_OK) return fail(nullptr, st, why);
    return MFC_OK;
}

MFC_API mfc_status mfc_destroy_lattice(mfc_lattice *L)
{
    if (!L) return MFC_ERR_ARG;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != L->device) cudaSetDevice(L->device);
    if (L->stream) cudaStreamSynchronize(L->stream);
    release(L);
    if (cur >= 0 && cur != L->device) cudaSetDevice(cur);
    delete L;
    return MFC_OK;
}

MFC_API mfc_status mfc_set_params(mfc_lattice *L, const mfc_params *params)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    std::string why;
    st = check_params(params, &why);
    if (st != MFC_OK) return fail(L, st, why);
    L->prm = *params;
    drop_graphs(L);  // the graphs hold the old constants
    return fill_ghosts(L);  // inlet and outlet ghost values depend on the parameters
}

MFC_API mfc_status mfc_set_geometry(mfc_lattice *L, const uint8_t *node_class, int reset_fields)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (!node_class) return fail(L, MFC_ERR_ARG, "node_class is NULL");
    for (long long q = 0; q < L->N; ++q)
        if (node_class[q] > 7) return fail(L, MFC_ERR_ARG, "node class above 7 at node " + std::to_string(q));
    CK(L, cudaMemcpyAsync(L->cls_tmp, node_class, (size_t)L->N, cudaMemcpyHostToDevice, L->stream));
    return apply_geometry(L, L->cls_tmp, reset_fields != 0);
}

static mfc_status step_n(mfc_lattice *L, int kind, int nsteps)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (nsteps < 0) return fail(L, MFC_ERR_ARG, "nsteps < 0");
    for (int s = 0; s < nsteps; ++s) {
        st = enqueue_step(L, kind, s == nsteps - 1 ? MODE_WRITE : MODE_PLAIN);
        if (st != MFC_OK) return st;
    }
    return MFC_OK;
}

MFC_API mfc_status mfc_step_flow(mfc_lattice *L, int nsteps) { return step_n(L, KIND_FLOW, nsteps); }
MFC_API mfc_status mfc_step_ade(mfc_lattice *L, int nsteps) { return step_n(L, KIND_ADE, nsteps); }
MFC_API mfc_status mfc_step_coupled(mfc_lattice *L, int nsteps) { return step_n(L, KIND_COUPLED, nsteps); }

MFC_API mfc_status mfc_step_coupled_plain(mfc_lattice *L, int nsteps)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (nsteps < 0) return fail(L, MFC_ERR_ARG, "nsteps < 0");
    for (int s = 0; s < nsteps; ++s) {
        st = enqueue_step(L, KIND_COUPLED, MODE_PLAIN);
        if (st != MFC_OK) return st;
    }
    return MFC_OK;
}

MFC_API mfc_status mfc_solve_steady(mfc_lattice *L, const mfc_solve_opts *opts, mfc_solve_result *out)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (!opts) return fail(L, MFC_ERR_ARG, "opts is NULL");
    if (opts->max_steps < 0 || opts->check_every < 1 || !(opts->tol_flow >= 0.0) ||
        !(opts->tol_ade >= 0.0) || (opts->mode != MFC_SEQUENTIAL && opts->mode != MFC_CONCURRENT))
        return fail(L, MFC_ERR_ARG, "bad solve options");
    const int K = opts->check_every;
    const double deadline = opts->timeout_s > 0.0 ? now_s() + opts->timeout_s : 0.0;
    mfc_solve_result r;
    memset(&r, 0, sizeof r);
    bool conv_f = false, conv_a = false;
    if (opts->mode == MFC_SEQUENTIAL) {
        double dummy = 0.0;
        st = run_phase(L, KIND_FLOW, opts->tol_flow, 0.0, opts->max_steps, K, deadline, &r.steps_flow,
                       &r.res_flow, &dummy, &conv_f);
        r.mass = L->results_h[SUM_MASS];
        if (st == MFC_OK)
            st = run_phase(L, KIND_ADE, 0.0, opts->tol_ade, opts->max_steps, K, deadline, &r.steps_ade,
                           &dummy, &r.res_ade, &conv_a);
    } else {
        st = run_phase(L, KIND_COUPLED, opts->tol_flow, opts->tol_ade, opts->max_steps, K, deadline,
                       &r.steps_flow, &r.res_flow, &r.res_ade, &conv_f);
        r.steps_ade = r.steps_flow;
        r.mass = L->results_h[SUM_MASS];
        conv_a = conv_f;
    }
    r.current = L->results_h[SUM_CURRENT];
    r.substrate = L->results_h[SUM_C];
    if (st != MFC_ERR_CUDA) {
        const mfc_status bs = check_bounds(L);
        if (bs != MFC_OK) st = bs;
    }
    if (st == MFC_OK && !(conv_f && conv_a)) st = MFC_NOT_CONVERGED;
    r.status = st;
    if (out) *out = r;
    return st;
}

MFC_API mfc_status mfc_step_check_sums(mfc_lattice *L, int nsteps, double *sums)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (nsteps < 1 || !sums) return fail(L, MFC_ERR_ARG, "nsteps must be >= 1 and sums non-NULL");
    st = enqueue_block(L, KIND_COUPLED, nsteps, true);
    if (st != MFC_OK) return st;
    CK(L, cudaStreamSynchronize(L->stream));
    st = check_bounds(L);
    if (st != MFC_OK) return st;
    for (int m = 0; m < NSUM; ++m) sums[m] = L->results_h[m];
    L->last_current = L->results_h[SUM_CURRENT];
    return MFC_OK;
}

MFC_API mfc_status mfc_set_halo_classes(mfc_lattice *L, int side, const uint8_t *plane)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if ((side != 0 && side != 1) || !plane) return fail(L, MFC_ERR_ARG, "side must be 0 or 1, plane non-NULL");
    if (!L->desc.cut[side]) return fail(L, MFC_ERR_STATE, "that face is not a cut");
    const size_t n = L->dim == 2 ? (size_t)L->ny : (size_t)L->nx * L->ny;
    for (size_t q = 0; q < n; ++q)
        if (plane[q] > 7) return fail(L, MFC_ERR_ARG, "class values above 7");
    if (!L->halo_cls[side]) {
        void *p = nullptr;
        if (!dev_alloc(L, &p, round_up(n, 256))) return fail(L, MFC_ERR_OOM, "halo classes: allocation failed");
        L->halo_cls[side] = static_cast<uint8_t *>(p);
        L->bytes += round_up(n, 256);
    }
    CK(L, cudaMemcpyAsync(L->halo_cls[side], plane, n, cudaMemcpyHostToDevice, L->stream));
    return apply_geometry(L, L->cls_cur, 0);
}

MFC_API mfc_status mfc_biofilm_grow(mfc_lattice *L, uint64_t seed, uint64_t cycle, double prob,
                                    double c_thresh, long *n_converted)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (!(prob >= 0.0 && prob <= 1.0) || !isfinite(c_thresh))
        return fail(L, MFC_ERR_ARG, "prob must be in [0,1], c_thresh finite");
    GrowArgs g;
    memset(&g, 0, sizeof g);
    g.geo = L->geo;
    g.cls = L->cls_cur;
    g.cls_out = L->cls_tmp;
    g.fld_c = L->fld_c;
    g.dbl = L->dbl;
    g.c_ref = L->c_ref;
    g.c_thresh = c_thresh;
    g.seed = seed;
    g.cycle = cycle;
    g.lim = (uint64_t)floor(prob * 9007199254740992.0);
    g.count = L->counts_d;
    CK(L, cudaMemsetAsync(L->counts_d, 0, sizeof(unsigned long long), L->stream));
    CK(L, launch_grow(L->dim, g, L->stream));
    CK(L, cudaMemcpyAsync(L->counts_h, L->counts_d, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          L->stream));
    CK(L, cudaStreamSynchronize(L->stream));
    const long n = (long)L->counts_h[0];
    st = apply_geometry(L, L->cls_tmp, 0);
    if (st != MFC_OK) return st;
    if (n_converted) *n_converted = n;
    return MFC_OK;
}

MFC_API mfc_status mfc_read_fields(mfc_lattice *L, double *rho, double *u, double *c, double *current)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    st = lattice_fields_async(L, rho, u, c);
    if (st != MFC_OK) return st;
    CK(L, cudaStreamSynchronize(L->stream));
    st = check_bounds(L);
    if (st != MFC_OK) return st;
    if (current) *current = L->last_current;
    return MFC_OK;
}



static mfc_status pop_io(mfc_lattice *L, int which, double *host_out, const double *host_in)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (!host_out && !host_in) return fail(L, MFC_ERR_ARG, "host buffer is NULL");
    PopArgs a;
    memset(&a, 0, sizeof a);
    a.geo = L->geo;
    a.link = L->link;
    a.link32 = L->link32;
    if (which == MFC_POP_FLOW) {
        a.q = L->qf;
        a.pop = L->f[L->fcur];
        a.half = L->half;
        a.dbl = L->dbl;
        a.self_bit = 0;
        a.offset = 1.0;
        for (int i = 0; i < a.q; ++i)
            a.w[i] = L->dim == 2 ? (L->dbl ? FlowSet<2>::wd(i) : FlowSet<2>::w(i))
                                 : (L->dbl ? FlowSet<3>::wd(i) : FlowSet<3>::w(i));
    } else if (which == MFC_POP_ADE) {
        a.q = L->qa;
        a.pop = L->g[L->gcur];
        a.half = L->half;
        a.dbl = L->dbl;
        a.self_bit = L->qf;
        a.offset = L->c_ref;
        for (int i = 0; i < a.q; ++i) {
            if (L->dbl) a.w[i] = L->qa == 9 ? AdeSet<2, 9>::wd(i) : (L->dim == 2 ? AdeSet<2>::wd(i) : AdeSet<3>::wd(i));
            else a.w[i] = L->qa == 9 ? AdeSet<2, 9>::w(i) : (L->dim == 2 ? AdeSet<2>::w(i) : AdeSet<3>::w(i));
        }
    } else if (which == MFC_FIELD_VELOCITY) {
        a.q = L->dim;
        a.pop = L->fld_u;
        a.half = 0;
        a.dbl = L->dbl;
        a.self_bit = host_out ? 0 : -1;
        a.offset = 0.0f;
    } else {
        return fail(L, MFC_ERR_ARG, "unknown population kind");
    }
    const size_t bytes = (size_t)a.q * L->N * sizeof(double);
    st = ensure_staging(L, bytes);
    if (st != MFC_OK) return st;
    a.dense = L->staging;
    a.to_dense = host_out != nullptr;
    if (host_in) CK(L, cudaMemcpyAsync(L->staging, host_in, bytes, cudaMemcpyHostToDevice, L->stream));
    CK(L, launch_pop_convert(a, L->stream));
    if (host_out) CK(L, cudaMemcpyAsync(host_out, L->staging, bytes, cudaMemcpyDeviceToHost, L->stream));
    if (host_in && which != MFC_FIELD_VELOCITY) {
        st = fill_ghosts(L);
        if (st != MFC_OK) return st;
    }
    CK(L, cudaStreamSynchronize(L->stream));
    return check_bounds(L);
}

MFC_API mfc_status mfc_read_populations(mfc_lattice *L, int which, double *host)
{
    return pop_io(L, which, host, nullptr);
}

MFC_API mfc_status mfc_write_populations(mfc_lattice *L, int which, const double *host)
{
    return pop_io(L, which, nullptr, host);
}

MFC_API mfc_status mfc_synchronize(mfc_lattice *L)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    CK(L, cudaStreamSynchronize(L->stream));
    return check_bounds(L);
}

#ifdef MFC_CHECK_BOUNDS
// Bytes of the guard regions [p, p + n) that differ from the pattern, added to *bad.
__global__ void guard_count_kernel(const unsigned char *p, size_t n, unsigned long long *bad)
{
    unsigned long long c = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        c += p[i] != GUARD_BYTE;
    if (c) atomicAdd(bad, c);
}
#endif

MFC_API mfc_status mfc_check_canaries(mfc_lattice *L, long long *bad)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (!bad) return fail(L, MFC_ERR_ARG, "bad is NULL");
    *bad = 0;
#ifdef MFC_CHECK_BOUNDS
    CK(L, cudaStreamSynchronize(L->stream));
    CK(L, cudaMemsetAsync(L->counts_d, 0, sizeof(unsigned long long), L->stream));
    for (auto &g : L->guards) {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(g.first);
        guard_count_kernel<<<1, 256, 0, L->stream>>>(b, GUARD, L->counts_d);
        guard_count_kernel<<<1, 256, 0, L->stream>>>(b + GUARD + g.second, GUARD, L->counts_d);
    }
    CK(L, cudaGetLastError());
    unsigned long long n = 0;
    CK(L, cudaMemcpyAsync(&n, L->counts_d, sizeof n, cudaMemcpyDeviceToHost, L->stream));
    CK(L, cudaStreamSynchronize(L->stream));
    *bad = (long long)n;
#endif
    return MFC_OK;
}

MFC_API int mfc_check_build(void)
{
#ifdef MFC_CHECK_BOUNDS
    return 1;
#else
    return 0;
#endif
}

MFC_API mfc_status mfc_set_launch(mfc_lattice *L, const mfc_launch *v)
{
    mfc_status st = enter(L);
    if (st != MFC_OK) return st;
    if (!v) return fail(L, MFC_ERR_ARG, "launch is NULL");
    if (v->block != 128 && v->block != 256) return fail(L, MFC_ERR_ARG, "block must be 128 or 256");
    if (v->offsets32 != 0 && v->offsets32 != 1) return fail(L, MFC_ERR_ARG, "offsets32 must be 0 or 1");
    CK(L, cudaStreamSynchronize(L->stream));
    L->block = v->block;
    L->offsets32 = v->offsets32;
    choose_launch(L);
    drop_graphs(L);
    return MFC_OK;
}

MFC_API mfc_status mfc_get_launch(mfc_lattice *L, mfc_launch *v)
{
    if (!L || !v) return MFC_ERR_ARG;
    v->block = L->block;
    v->offsets32 = L->offsets32;
    return MFC_OK;
}

MFC_API mfc_status mfc_active_nodes(mfc_lattice *L, long *flow_open, long *ade_open)
{
    if (!L) return MFC_ERR_ARG;
    if (flow_open) *flow_open = L->flow_open;
    if (ade_open) *ade_open = L->ade_open;
    return MFC_OK;
}

MFC_API mfc_status mfc_device_bytes(mfc_lattice *L, size_t *bytes)
{
    if (!L || !bytes) return MFC_ERR_ARG;
    *bytes = L->bytes + L->staging_bytes;
    return MFC_OK;
}

MFC_API const char *mfc_status_string(mfc_status s)
{
    switch (s) {
    case MFC_OK: return "ok";
    case MFC_ERR_ARG: return "invalid argument";
    case MFC_ERR_OOM: return "out of device memory";
    case MFC_ERR_OOM_BUDGET: return "over the memory budget";
    case MFC_ERR_CUDA: return "CUDA error";
    case MFC_NOT_CONVERGED: return "not converged within the step cap";
    case MFC_ERR_NONFINITE: return "non-finite residual, mass or current";
    case MFC_ERR_UNSTABLE: return "flow at or above the lattice sound speed, or non-positive density";
    case MFC_ERR_TIMEOUT: return "wall-clock limit reached";
    case MFC_ERR_STATE: return "invalid state";
    case MFC_PENDING: return "pending";
    }
    return "unknown status";
}

MFC_API const char *mfc_last_error(mfc_lattice *L)
{
    return L ? L->err.c_str() : g_create_error.c_str();
}

MFC_API const char *mfc_version(void) { return "mfc 0.1 sm_103a"; }

}  // extern "C"
