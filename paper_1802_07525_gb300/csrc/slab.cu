// Halo exchange of the slab decomposition: one lattice split along its flow axis into slabs whose
// faces towards each other are cuts.  The populations that leave a slab through a cut face are
// those of the layer next to it along the directions pointing out of it (pull scheme: the
// neighbour's first layer pulls them from its ghost layer).  Pack copies them, direction by
// direction, into a dense buffer; unpack writes a neighbour's buffer into the ghost layer, with
// the periodic images of the cross axes in the ghost ring, where pulls along the diagonals find
// them.  Values move in their storage type, so the slabs compute what the whole lattice does.
#include <string.h>

#include <string>

#include "lbm_kernels.cuh"
#include "runtime.h"

using namespace mfc;

namespace {

struct HaloArgs {
    Geo geo;
    int dim;
    int bc[3];
    int side;            // 0: low face of the flow axis, 1: high face
    int nf, na;          // crossing flow / transport planes
    int fplane[19], aplane[9];
    const void *fpop;    // flow populations (current buffer)
    const void *gpop;    // transport populations (current buffer)
    void *fpop_w, *gpop_w;
    void *buf;
};

// Planes of a velocity set along which populations cross face `side` going out (out = true) or
// coming in.
template <typename SET> int crossing(int fa, int side, bool out, int *planes)
{
    const int want = (side == 0) == out ? -1 : 1;
    int n = 0;
    for (int i = 1; i < SET::Q; ++i)
        if (SET::c(i, fa) == want) planes[n++] = i;
    return n;
}

__device__ __forceinline__ long long cross_count(const HaloArgs &a)
{
    return a.dim == 2 ? (long long)a.geo.ny : (long long)a.geo.nx * a.geo.ny;
}

// element of cross-section position c (dense) in the layer with flow-axis coordinate f
__device__ __forceinline__ long long layer_elem(const HaloArgs &a, long long c, int f)
{
    if (a.dim == 2) return a.geo.at(f, (int)c, 0);
    return a.geo.at((int)(c % a.geo.nx), (int)(c / a.geo.nx), f);
}

template <typename T> __global__ void halo_pack_kernel(const HaloArgs a)
{
    const long long C = cross_count(a);
    const int nfa = a.dim == 2 ? a.geo.nx : a.geo.nz;
    const int f = a.side == 0 ? 0 : nfa - 1;
    const long long total = (long long)(a.nf + a.na) * C;
    T *out = static_cast<T *>(a.buf);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(q / C);
        const long long c = q - (long long)p * C;
        const long long k = layer_elem(a, c, f);
        out[q] = p < a.nf ? static_cast<const T *>(a.fpop)[(long long)a.fplane[p] * a.geo.plane + k]
                          : static_cast<const T *>(a.gpop)[(long long)a.aplane[p - a.nf] * a.geo.plane + k];
    }
}

// Ghost-layer cells of face `side`, the ring included: the cross coordinates run over
// [-1, n] on each cross axis; a ring cell takes its periodic image's value (walls: no value needed,
// the links across them bounce back).
template <typename T> __global__ void halo_unpack_kernel(const HaloArgs a)
{
    const long long C = cross_count(a);
    const int nfa = a.dim == 2 ? a.geo.nx : a.geo.nz;
    const int f = a.side == 0 ? -1 : nfa;
    const int w0 = a.dim == 2 ? a.geo.ny + 2 : a.geo.nx + 2;  // ring-inclusive extents
    const int w1 = a.dim == 2 ? 1 : a.geo.ny + 2;
    const long long ring = (long long)w0 * w1;
    const long long total = (long long)(a.nf + a.na) * ring;
    const T *in = static_cast<const T *>(a.buf);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(q / ring);
        const long long r = q - (long long)p * ring;
        int c0 = (int)(r % w0) - 1, c1 = a.dim == 2 ? 0 : (int)(r / w0) - 1;
        // cross axes: 2-D y (axis 1); 3-D x and y (axes 0, 1)
        const int ax0 = a.dim == 2 ? 1 : 0;
        const int n0 = a.dim == 2 ? a.geo.ny : a.geo.nx;
        int s0 = c0, s1 = c1;
        bool ok = true;
        if (s0 < 0 || s0 >= n0) {
            if (a.bc[ax0] == BC_PERIODIC) s0 = s0 < 0 ? s0 + n0 : s0 - n0;
            else ok = false;
        }
        if (a.dim == 3 && (s1 < 0 || s1 >= a.geo.ny)) {
            if (a.bc[1] == BC_PERIODIC) s1 = s1 < 0 ? s1 + a.geo.ny : s1 - a.geo.ny;
            else ok = false;
        }
        if (!ok) continue;
        const long long c = a.dim == 2 ? (long long)s0 : s0 + (long long)a.geo.nx * s1;
        const long long k = a.dim == 2 ? a.geo.at(f, c0, 0) : a.geo.at(c0, c1, f);
        const T v = in[(long long)p * C + c];
        if (p < a.nf) static_cast<T *>(a.fpop_w)[(long long)a.fplane[p] * a.geo.plane + k] = v;
        else static_cast<T *>(a.gpop_w)[(long long)a.aplane[p - a.nf] * a.geo.plane + k] = v;
    }
}

mfc_status halo_args(mfc_lattice *L, int side, bool out, HaloArgs *a)
{
    mfc_status st = lattice_enter(L);
    if (st != MFC_OK) return st;
    if (side != 0 && side != 1) return lattice_fail(L, MFC_ERR_ARG, "side must be 0 or 1");
    if (!L->desc.cut[side]) return lattice_fail(L, MFC_ERR_STATE, "that face is not a cut");
    memset(a, 0, sizeof *a);
    a->geo = L->geo;
    a->dim = L->dim;
    for (int i = 0; i < 3; ++i) a->bc[i] = i < L->dim ? L->desc.bc[i] : BC_PERIODIC;
    a->side = side;
    const int fa = L->dim == 2 ? 0 : 2;
    if (L->dim == 2) {
        a->nf = crossing<FlowSet<2>>(fa, side, out, a->fplane);
        a->na = L->qa == 9 ? crossing<AdeSet<2, 9>>(fa, side, out, a->aplane)
                           : crossing<AdeSet<2, 5>>(fa, side, out, a->aplane);
    } else {
        a->nf = crossing<FlowSet<3>>(fa, side, out, a->fplane);
        a->na = crossing<AdeSet<3, 7>>(fa, side, out, a->aplane);
    }
    a->fpop = L->f[L->fcur];
    a->gpop = L->g[L->gcur];
    a->fpop_w = L->f[L->fcur];
    a->gpop_w = L->g[L->gcur];
    return MFC_OK;
}

int grid_of(long long n)
{
    const long long b = (n + 255) / 256;
    return (int)(b < 2048 ? (b > 0 ? b : 1) : 2048);
}

}  // namespace

extern "C" MFC_API mfc_status mfc_halo_bytes(mfc_lattice *L, int side, size_t *bytes)
{
    HaloArgs a;
    mfc_status st = halo_args(L, side, true, &a);
    if (st != MFC_OK) return st;
    if (!bytes) return lattice_fail(L, MFC_ERR_ARG, "bytes is NULL");
    const size_t C = L->dim == 2 ? (size_t)L->ny : (size_t)L->nx * L->ny;
    *bytes = (size_t)(a.nf + a.na) * C * L->st_bytes;
    return MFC_OK;
}

extern "C" MFC_API mfc_status mfc_halo_pack(mfc_lattice *L, int side, void *dev_buf)
{
    HaloArgs a;
    mfc_status st = halo_args(L, side, true, &a);
    if (st != MFC_OK) return st;
    if (!dev_buf) return lattice_fail(L, MFC_ERR_ARG, "buffer is NULL");
    a.buf = dev_buf;
    const long long C = L->dim == 2 ? (long long)L->ny : (long long)L->nx * L->ny;
    const int g = grid_of((long long)(a.nf + a.na) * C);
    if (L->st_bytes == 2) halo_pack_kernel<uint16_t><<<g, 256, 0, L->stream>>>(a);
    else if (L->st_bytes == 4) halo_pack_kernel<uint32_t><<<g, 256, 0, L->stream>>>(a);
    else halo_pack_kernel<unsigned long long><<<g, 256, 0, L->stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lattice_fail(L, MFC_ERR_CUDA, std::string("halo pack: ") + cudaGetErrorString(e));
    return MFC_OK;
}

extern "C" MFC_API mfc_status mfc_halo_unpack(mfc_lattice *L, int side, const void *dev_buf)
{
    HaloArgs a;
    mfc_status st = halo_args(L, side, false, &a);
    if (st != MFC_OK) return st;
    if (!dev_buf) return lattice_fail(L, MFC_ERR_ARG, "buffer is NULL");
    a.buf = const_cast<void *>(dev_buf);
    const long long ring = L->dim == 2 ? (long long)L->ny + 2 : (long long)(L->nx + 2) * (L->ny + 2);
    const int g = grid_of((long long)(a.nf + a.na) * ring);
    if (L->st_bytes == 2) halo_unpack_kernel<uint16_t><<<g, 256, 0, L->stream>>>(a);
    else if (L->st_bytes == 4) halo_unpack_kernel<uint32_t><<<g, 256, 0, L->stream>>>(a);
    else halo_unpack_kernel<unsigned long long><<<g, 256, 0, L->stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lattice_fail(L, MFC_ERR_CUDA, std::string("halo unpack: ") + cudaGetErrorString(e));
    return MFC_OK;
}
