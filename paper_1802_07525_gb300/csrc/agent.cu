// Agent-based biofilm formation between steady solves (Tsompanas et al., arXiv 1802.07525,
// Sec. 3.3): attachment of k_ata front cells, growth by the double Monod law (Eq. 16) and
// spreading of biomass above C_max^bio, on a per-node biomass concentration held on the device.
//
// Attachment and growth are data-parallel.  The exact choice of the k_ata front cells with the
// smallest keys is a radix selection on the device (eight 8-bit digits of unique 64-bit keys:
// per-block shared-memory histograms, then one small kernel that picks the digit).  Spreading
// moves biomass along chains, one event after another, each event seeing the previous ones, so
// it runs as a single device thread over the ordered list of cells above the threshold (compacted
// in order by one block); a walk's path membership is an O(1) mark per node.  Every loop of the
// serial kernel is bounded (events by the list, steps by max_walk).
#include <math.h>
#include <string.h>

#include <string>

#include "lbm_kernels.cuh"
#include "runtime.h"

using namespace mfc;

namespace {

// splitmix64 of Steele, Lea and Flood (OOPSLA 2014), as published by Vigna.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// (x, y, z) of dense node q (x fastest).
__device__ __forceinline__ void xyz_of(const Geo &g, long long q, int *x, int *y, int *z)
{
    const long long row = q / g.nx;
    *x = (int)(q - row * g.nx);
    *y = (int)(row % g.ny);
    *z = (int)(row / g.ny);
}

constexpr unsigned long long NO_KEY = ~0ull;
constexpr uint64_t ATTACH_TAG = 0x6174746163680000ull;  // "attach"
constexpr uint64_t SPREAD_TAG = 0x7370726561640000ull;  // "spread"
constexpr uint8_t ELECTRODE = CLS_FLOW | CLS_ADE;

enum : int { ST_ATTACHED = 0, ST_FRONT, ST_SPREAD, ST_FAILED, ST_STEPS, ST_BIOFILM, ST_NLIST, ST_N };

// Device-side state of one call: the radix selection and the statistics.
struct AgentState {
    unsigned long long prefix, mask;
    unsigned int k_rem, all;
    unsigned int hist[256];
    unsigned long long count[ST_N];
    double total;
};

struct AgentArgs {
    Geo geo;
    const uint8_t *cls;
    uint8_t *cls_out;
    double *bio;
    const void *fld_c;  // C - c_ref (pitched), FP32 or FP64
    int dbl;
    float c_ref;
    unsigned long long *keys;
    int *list, *mark, *path;
    AgentState *st;
    uint64_t attach_base, spread_base, cycle;
    double c0, cmax, fr, mu, ks;
    int max_walk;
};

__device__ __forceinline__ bool in_lattice(const Geo &g, int x, int y, int z)
{
    return x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz;
}

__device__ __forceinline__ long long dense(const Geo &g, int x, int y, int z)
{
    return x + (long long)g.nx * (y + (long long)g.ny * z);
}

// Substrate concentration of node q as mfc_read_fields reports it for a transport-open node.
__device__ __forceinline__ double conc_at(const AgentArgs &a, int x, int y, int z)
{
    const long long k = a.geo.at(x, y, z);
    return a.dbl ? (double)a.c_ref + reinterpret_cast<const double *>(a.fld_c)[k]
                 : (double)(a.c_ref + reinterpret_cast<const float *>(a.fld_c)[k]);
}

template <int DIM> __global__ void agent_keys_kernel(const AgentArgs a)
{
    using F = FlowSet<DIM>;
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        unsigned long long key = NO_KEY;
        if (a.cls[q] == 0 && a.bio[q] == 0.0) {
            int x, y, z;
            xyz_of(a.geo, q, &x, &y, &z);
            bool front = false;
#pragma unroll
            for (int i = 1; i < F::Q; ++i) {
                const int sx = x + F::c(i, 0), sy = y + F::c(i, 1), sz = z + F::c(i, 2);
                if (in_lattice(a.geo, sx, sy, sz) && (a.cls[dense(a.geo, sx, sy, sz)] & ELECTRODE) == ELECTRODE)
                    front = true;
            }
            if (front) {
                const uint64_t h = mix64(a.attach_base ^ (a.cycle << 32) ^ (uint64_t)q);
                key = ((h >> 32) << 32) | (uint64_t)(uint32_t)q;
                atomicAdd(&a.st->count[ST_FRONT], 1ull);
            }
        }
        a.keys[q] = key;
    }
}

__global__ void agent_select_init_kernel(AgentState *st, unsigned int k)
{
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->mask = 0;
        st->k_rem = k;
        st->all = 0;
        st->total = 0.0;
    }
    for (int b = threadIdx.x; b < 256; b += blockDim.x) st->hist[b] = 0;
    for (int m = threadIdx.x; m < ST_N; m += blockDim.x) st->count[m] = 0;
}

// Histogram of digit `shift` of the keys that match the selected prefix.
__global__ void __launch_bounds__(256) agent_hist_kernel(const unsigned long long *keys, long long N, AgentState *st,
                                                         int shift)
{
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long prefix = st->prefix, mask = st->mask;
    if (!st->all) {
        for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
             q += (long long)gridDim.x * blockDim.x) {
            const unsigned long long k = keys[q];
            if (k != NO_KEY && (k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

// Fix digit `shift` of the k-th smallest key: the digit whose bucket holds the k_rem-th key.
__global__ void agent_pick_kernel(AgentState *st, int shift)
{
    if (threadIdx.x == 0 && !st->all) {
        unsigned int cum = 0;
        int d = -1;
        for (int b = 0; b < 256; ++b) {
            if (cum + st->hist[b] >= st->k_rem) {
                d = b;
                break;
            }
            cum += st->hist[b];
        }
        if (d < 0) {
            st->all = 1;  // fewer keys than asked for: every front node attaches
        } else {
            st->prefix |= (unsigned long long)d << shift;
            st->mask |= 255ull << shift;
            st->k_rem -= cum;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) st->hist[b] = 0;
}

// Attachment, then growth (Eq. 16), node by node.
__global__ void agent_attach_grow_kernel(const AgentArgs a, int select)
{
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    const unsigned long long T = a.st->prefix;  // the k-th smallest key
    const bool all = a.st->all != 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
         q += (long long)gridDim.x * blockDim.x) {
        double b = a.bio[q];
        const unsigned long long key = a.keys[q];
        if (select && key != NO_KEY && (all || key <= T)) {
            b = a.c0;
            atomicAdd(&a.st->count[ST_ATTACHED], 1ull);
        }
        if (b > 0.0 && !(a.cls[q] & CLS_ADE)) {
            int x, y, z;
            xyz_of(a.geo, q, &x, &y, &z);
            double C = conc_at(a, x, y, z);
            C = C > 0.0 ? C : 0.0;
            // b (1 + mu C / (C + K_s)), each operation rounded once (no contraction)
            b = __dmul_rn(b, __dadd_rn(1.0, __dmul_rn(a.mu, __ddiv_rn(C, __dadd_rn(C, a.ks)))));
        }
        a.bio[q] = b;
    }
}

// The nodes above C_max^bio (not electrode), in increasing order: one block, ordered compaction.
__global__ void __launch_bounds__(1024) agent_list_kernel(const AgentArgs a)
{
    __shared__ int warp_off[32];
    __shared__ int base, chunk;
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (long long q0 = 0; q0 < N; q0 += blockDim.x) {
        const long long q = q0 + threadIdx.x;
        const bool flag = q < N && a.bio[q] > a.cmax && !(a.cls[q] & CLS_ADE);
        const unsigned int m = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) warp_off[warp] = __popc(m);
        __syncthreads();
        if (warp == 0) {
            const int nw = (int)(blockDim.x >> 5);
            const int v = lane < nw ? warp_off[lane] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane < nw) warp_off[lane] = incl - v;
            if (lane == 31) chunk = incl;
        }
        __syncthreads();
        if (flag) a.list[base + warp_off[warp] + __popc(m & ((1u << lane) - 1u))] = (int)q;
        __syncthreads();
        if (threadIdx.x == 0) base += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.st->count[ST_NLIST] = (unsigned long long)base;
}

// Spreading: one thread, events in list order.
template <int DIM> __global__ void agent_spread_kernel(const AgentArgs a)
{
    using F = FlowSet<DIM>;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const Geo &g = a.geo;
    const long long nl = (long long)a.st->count[ST_NLIST];
    unsigned long long nd = 0, spread = 0, failed = 0, steps = 0;
    for (long long e = 0; e < nl; ++e) {
        const int k = a.list[e];
        if (!(a.bio[k] > a.cmax)) continue;
        int x, y, z;
        xyz_of(g, k, &x, &y, &z);
        int freen[F::Q];
        int nfree = 0;
        for (int i = 1; i < F::Q; ++i) {
            const int sx = x + F::c(i, 0), sy = y + F::c(i, 1), sz = z + F::c(i, 2);
            if (!in_lattice(g, sx, sy, sz)) continue;
            const int j = (int)dense(g, sx, sy, sz);
            if (!(a.cls[j] & ELECTRODE) && a.bio[j] == 0.0) freen[nfree++] = j;
        }
        int target;
        if (nfree > 0) {
            const uint64_t d = mix64(a.spread_base ^ nd++);
            target = freen[(d >> 32) % (uint64_t)nfree];
        } else {
            // loop-erased random walk from k; mark[j] is j's position on the path
            int len = 1;
            a.path[0] = k;
            a.mark[k] = 0;
            bool found = false;
            for (int s = 0; s < a.max_walk && !found; ++s) {
                ++steps;
                const uint64_t d = mix64(a.spread_base ^ nd++);
                const int i = 1 + (int)((d >> 32) % (uint64_t)(F::Q - 1));
                int cx, cy, cz;
                xyz_of(g, a.path[len - 1], &cx, &cy, &cz);
                const int sx = cx + F::c(i, 0), sy = cy + F::c(i, 1), sz = cz + F::c(i, 2);
                if (!in_lattice(g, sx, sy, sz)) continue;
                const int j = (int)dense(g, sx, sy, sz);
                if (a.cls[j] & CLS_ADE) continue;  // electrode: the step is lost
                const int at = a.mark[j];
                if (at >= 0) {  // back onto the path: erase the loop
                    for (int m = at + 1; m < len; ++m) a.mark[a.path[m]] = -1;
                    len = at + 1;
                    continue;
                }
                a.mark[j] = len;
                a.path[len++] = j;
                if (a.bio[j] == 0.0) found = true;
            }
            for (int m = 0; m < len; ++m) a.mark[a.path[m]] = -1;
            if (!found) {
                ++failed;
                continue;
            }
            for (int m = len - 1; m >= 2; --m) a.bio[a.path[m]] = a.bio[a.path[m - 1]];
            target = a.path[1];
            a.bio[target] = 0.0;
        }
        const double t = __dmul_rn(a.fr, a.bio[k]);
        a.bio[k] = __dadd_rn(a.bio[k], -t);
        a.bio[target] = t;
        ++spread;
    }
    a.st->count[ST_SPREAD] = spread;
    a.st->count[ST_FAILED] = failed;
    a.st->count[ST_STEPS] = steps;
}

// Classes after the step, and the biofilm statistics (one block, a fixed order of addition).
__global__ void __launch_bounds__(256) agent_classes_kernel(const AgentArgs a)
{
    const long long N = (long long)a.geo.nx * a.geo.ny * a.geo.nz;
    double tot = 0.0;
    unsigned long long nb = 0;
    for (long long q = threadIdx.x; q < N; q += blockDim.x) {
        const double b = a.bio[q];
        const uint8_t c = a.cls[q];
        a.cls_out[q] = (b > 0.0 && !(c & CLS_ADE)) ? (uint8_t)(CLS_FLOW | CLS_SINK) : c;
        if (b > 0.0) ++nb;
        tot += b;
    }
    __shared__ double sh[256];
    __shared__ unsigned long long sn[256];
    sh[threadIdx.x] = tot;
    sn[threadIdx.x] = nb;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[threadIdx.x] += sh[threadIdx.x + s];
            sn[threadIdx.x] += sn[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.st->total = sh[0];
        a.st->count[ST_BIOFILM] = sn[0];
    }
}

#define ACK(L, call)                                                                            \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return lattice_fail(L, MFC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Device buffers of the agent model (biomass, keys, list, marks, state; the path grows with
// max_walk).  The marks start at -1.
mfc_status ensure_agent(mfc_lattice *L, int max_walk)
{
    const size_t N = (size_t)L->N;
    auto get = [&](void **p, size_t bytes) {
        if (*p) return true;
        if (!lattice_alloc(L, p, bytes)) return false;
        L->bytes += bytes;
        return true;
    };
    if (!get((void **)&L->biomass, N * sizeof(double)) ||
        !get((void **)&L->agent_keys, N * sizeof(unsigned long long)) ||
        !get((void **)&L->agent_list, N * sizeof(int)) || !get(&L->agent_state, sizeof(AgentState)))
        return lattice_fail(L, MFC_ERR_OOM, "agent buffers: device allocation failed");
    if (!L->agent_mark) {
        if (!get((void **)&L->agent_mark, N * sizeof(int)))
            return lattice_fail(L, MFC_ERR_OOM, "agent buffers: device allocation failed");
        ACK(L, cudaMemsetAsync(L->agent_mark, 0xff, N * sizeof(int), L->stream));
    }
    if (max_walk + 2 > L->agent_path_cap) {
        if (L->agent_path) {
            lattice_free(L, L->agent_path);
            L->agent_path = nullptr;
        }
        const int cap = max_walk + 2 > 1026 ? max_walk + 2 : 1026;
        if (!get((void **)&L->agent_path, (size_t)cap * sizeof(int)))
            return lattice_fail(L, MFC_ERR_OOM, "agent path: device allocation failed");
        L->agent_path_cap = cap;
    }
    return MFC_OK;
}

int grid_for(long long N)
{
    const long long b = (N + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

extern "C" MFC_API mfc_status mfc_agent_step(mfc_lattice *L, const mfc_agent_params *p, uint64_t cycle,
                                             mfc_agent_stats *out)
{
    mfc_status st = lattice_enter(L);
    if (st != MFC_OK) return st;
    if (!p) return lattice_fail(L, MFC_ERR_ARG, "agent parameters are NULL");
    if (p->k_ata < 0 || !(p->c0_bio > 0.0) || !isfinite(p->c0_bio) || !(p->c_max_bio > 0.0) ||
        !isfinite(p->c_max_bio) || !(p->fr_spr >= 0.0 && p->fr_spr <= 1.0) || !(p->growth >= 0.0) ||
        !isfinite(p->growth) || !(p->k_half > 0.0) || !isfinite(p->k_half) || p->max_walk < 1 ||
        p->max_walk > 65536)
        return lattice_fail(L, MFC_ERR_ARG, "agent parameters out of range");
    if (L->N >= (1ll << 31)) return lattice_fail(L, MFC_ERR_ARG, "agent model: lattice of 2^31 nodes or more");
    st = ensure_agent(L, p->max_walk);
    if (st != MFC_OK) return st;
    AgentArgs a;
    memset(&a, 0, sizeof a);
    a.geo = L->geo;
    a.cls = L->cls_cur;
    a.cls_out = L->cls_tmp;
    a.bio = L->biomass;
    a.fld_c = L->fld_c;
    a.dbl = L->dbl;
    a.c_ref = L->c_ref;
    a.keys = L->agent_keys;
    a.list = L->agent_list;
    a.mark = L->agent_mark;
    a.path = L->agent_path;
    a.st = static_cast<AgentState *>(L->agent_state);
    a.attach_base = mix64(p->seed ^ ATTACH_TAG);
    a.spread_base = mix64(p->seed ^ SPREAD_TAG ^ (cycle << 32));
    a.cycle = cycle;
    a.c0 = p->c0_bio;
    a.cmax = p->c_max_bio;
    a.fr = p->fr_spr;
    a.mu = p->growth;
    a.ks = p->k_half;
    a.max_walk = p->max_walk;
    const long long N = L->N;
    cudaStream_t s = L->stream;
    agent_select_init_kernel<<<1, 256, 0, s>>>(a.st, (unsigned int)p->k_ata);
    if (L->dim == 2) agent_keys_kernel<2><<<grid_for(N), 256, 0, s>>>(a);
    else agent_keys_kernel<3><<<grid_for(N), 256, 0, s>>>(a);
    if (p->k_ata > 0) {
        for (int shift = 56; shift >= 0; shift -= 8) {
            agent_hist_kernel<<<grid_for(N), 256, 0, s>>>(a.keys, N, a.st, shift);
            agent_pick_kernel<<<1, 256, 0, s>>>(a.st, shift);
        }
    }
    agent_attach_grow_kernel<<<grid_for(N), 256, 0, s>>>(a, p->k_ata > 0 ? 1 : 0);
    agent_list_kernel<<<1, 1024, 0, s>>>(a);
    if (L->dim == 2) agent_spread_kernel<2><<<1, 1, 0, s>>>(a);
    else agent_spread_kernel<3><<<1, 1, 0, s>>>(a);
    agent_classes_kernel<<<1, 256, 0, s>>>(a);
    ACK(L, cudaGetLastError());
    AgentState host;
    ACK(L, cudaMemcpyAsync(&host, a.st, sizeof host, cudaMemcpyDeviceToHost, s));
    ACK(L, cudaStreamSynchronize(s));
    st = lattice_apply_classes(L, L->cls_tmp, 0);
    if (st != MFC_OK) return st;
    if (out) {
        out->attached = (long long)host.count[ST_ATTACHED];
        out->front = (long long)host.count[ST_FRONT];
        out->spread = (long long)host.count[ST_SPREAD];
        out->walks_failed = (long long)host.count[ST_FAILED];
        out->walk_steps = (long long)host.count[ST_STEPS];
        out->biofilm_nodes = (long long)host.count[ST_BIOFILM];
        out->total_biomass = host.total;
    }
    return MFC_OK;
}

extern "C" MFC_API mfc_status mfc_read_biomass(mfc_lattice *L, double *host)
{
    mfc_status st = lattice_enter(L);
    if (st != MFC_OK) return st;
    if (!host) return lattice_fail(L, MFC_ERR_ARG, "host buffer is NULL");
    if (!L->biomass) {
        memset(host, 0, (size_t)L->N * sizeof(double));
        return MFC_OK;
    }
    ACK(L, cudaMemcpyAsync(host, L->biomass, (size_t)L->N * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    ACK(L, cudaStreamSynchronize(L->stream));
    return MFC_OK;
}

extern "C" MFC_API mfc_status mfc_write_biomass(mfc_lattice *L, const double *host)
{
    mfc_status st = lattice_enter(L);
    if (st != MFC_OK) return st;
    if (!host) return lattice_fail(L, MFC_ERR_ARG, "host buffer is NULL");
    for (long long q = 0; q < L->N; ++q)
        if (!(host[q] >= 0.0) || !isfinite(host[q])) return lattice_fail(L, MFC_ERR_ARG, "biomass must be finite and >= 0");
    if (L->N >= (1ll << 31)) return lattice_fail(L, MFC_ERR_ARG, "agent model: lattice of 2^31 nodes or more");
    st = ensure_agent(L, 1);
    if (st != MFC_OK) return st;
    ACK(L, cudaMemcpyAsync(L->biomass, host, (size_t)L->N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
    ACK(L, cudaStreamSynchronize(L->stream));
    return MFC_OK;
}
