// Residual, mass, substrate and current sums of two consecutive field snapshots, for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's memory pool or
// under a fixed device-memory budget, where a raw allocation would break the accounting or is
// forbidden, and code on a path that must not risk an allocation failure.  This entry point
// computes the sums of the check step of mfc_solve_steady (per-block partials added in a fixed
// order; here in FP64 throughout, on FP64 fields) on fields the caller already holds, and
// allocates nothing: its per-block partials live in the file-scope array below, which every GPU
// that loads the library holds until the process exits.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/mfc.h"

namespace {

constexpr int NA_BLOCK = 256;                 // nodes per block, one partial each
constexpr int NA_MAX_BLOCKS = 8192;           // partials the scratch holds
constexpr long long NA_MAX_NODES = (long long)NA_BLOCK * NA_MAX_BLOCKS;  // 2,097,152
constexpr int NA_NSUM = 8;
constexpr int NA_MAX_DEVICES = 64;

// 8192 blocks x 8 sums x 8 bytes = 512 KiB per device.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS * NA_NSUM];

std::mutex g_setup_mutex;
double *g_partials_addr[NA_MAX_DEVICES] = {};  // device address of the array, per device

__device__ __forceinline__ double na_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One block of NA_BLOCK nodes: the eight sums of the check step, reduced to one partial.
__global__ void __launch_bounds__(NA_BLOCK) na_sums_kernel(long long n, int dim, const uint8_t *cls,
                                                           const double *rho, const double *u,
                                                           const double *u_prev, const double *c,
                                                           const double *c_prev, double k_sink,
                                                           double *partials)
{
    double acc[NA_NSUM] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long q = (long long)blockIdx.x * NA_BLOCK + threadIdx.x;
    if (q < n) {
        const uint8_t k = cls[q];
        if (!(k & 1)) {  // open for the flow
            for (int a = 0; a < dim; ++a) {
                const double un = u[a * n + q], d = un - u_prev[a * n + q];
                acc[0] += d * d;
                acc[1] += un * un;
                if (!isfinite(un)) acc[7] += 1.0;
            }
            acc[2] += rho[q];
            if (!isfinite(rho[q])) acc[7] += 1.0;
        }
        if (!(k & 2)) {  // open for transport
            const double cn = c[q], d = cn - c_prev[q];
            acc[3] += d * d;
            acc[4] += cn * cn;
            acc[5] += cn;
            if (k & 4) acc[6] += k_sink * cn;
            if (!isfinite(cn)) acc[7] += 1.0;
        }
    }
    __shared__ double sh[NA_BLOCK / 32][NA_NSUM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int m = 0; m < NA_NSUM; ++m) acc[m] = na_warp_sum(acc[m]);
    if (lane == 0)
        for (int m = 0; m < NA_NSUM; ++m) sh[warp][m] = acc[m];
    __syncthreads();
    if (warp == 0) {
        for (int m = 0; m < NA_NSUM; ++m) {
            double v = lane < NA_BLOCK / 32 ? sh[lane][m] : 0.0;
            v = na_warp_sum(v);
            if (lane == 0) partials[(size_t)blockIdx.x * NA_NSUM + m] = v;
        }
    }
}

// Add the partials in a fixed order; write the eight sums and the two residuals.
__global__ void __launch_bounds__(256) na_finalize_kernel(const double *partials, int nblocks, double *out)
{
    __shared__ double sh[256][NA_NSUM];
    double acc[NA_NSUM] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int m = 0; m < NA_NSUM; ++m) acc[m] += partials[(size_t)b * NA_NSUM + m];
    for (int m = 0; m < NA_NSUM; ++m) sh[threadIdx.x][m] = acc[m];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int m = 0; m < NA_NSUM; ++m) sh[threadIdx.x][m] += sh[threadIdx.x + s][m];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int m = 0; m < NA_NSUM; ++m) out[m] = sh[0][m];
        const double du2 = sh[0][0], u2 = sh[0][1], dc2 = sh[0][3], c2 = sh[0][4];
        out[8] = u2 > 0.0 ? sqrt(du2 / u2) : (du2 > 0.0 ? INFINITY : 0.0);
        out[9] = c2 > 0.0 ? sqrt(dc2 / c2) : (dc2 > 0.0 ? INFINITY : 0.0);
    }
}

// Device address of the scratch array on the current device, looked up once per device.
mfc_status scratch_address(double **addr)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return MFC_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return MFC_ERR_CUDA;
        }
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    *addr = g_partials_addr[dev];
    return MFC_OK;
}

}  // namespace

extern "C" MFC_API mfc_status mfc_field_sums_noalloc(long long n, int dim, const uint8_t *node_class,
                                                      const double *rho, const double *u,
                                                      const double *u_prev, const double *c,
                                                      const double *c_prev, double k_sink,
                                                      double *out, void *stream)
{
    if (n < 1 || n > NA_MAX_NODES) return MFC_ERR_ARG;  // at most 2,097,152 nodes
    if (dim != 2 && dim != 3) return MFC_ERR_ARG;
    if (!node_class || !rho || !u || !u_prev || !c || !c_prev || !out) return MFC_ERR_ARG;
    double *partials = nullptr;
    mfc_status st = scratch_address(&partials);
    if (st != MFC_OK) return st;
    int nblocks = (int)((n + NA_BLOCK - 1) / NA_BLOCK);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Each launch reports its own error through its return value, so an error left pending by
    // earlier work of the caller is neither reported as this call's nor cleared.
    void *sums_args[] = {&n, &dim, &node_class, &rho, &u, &u_prev, &c, &c_prev, &k_sink, &partials};
    cudaError_t e = cudaLaunchKernel((const void *)na_sums_kernel, dim3((unsigned)nblocks), dim3(NA_BLOCK),
                                     sums_args, 0, s);
    if (e == cudaSuccess) {
        void *fin_args[] = {&partials, &nblocks, &out};
        e = cudaLaunchKernel((const void *)na_finalize_kernel, dim3(1), dim3(256), fin_args, 0, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();  // the launch failure just recorded by this call
        return MFC_ERR_CUDA;
    }
    return MFC_OK;
}
