// Host-side declarations shared by the runtime and the per-dimension kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"

namespace mfc {

enum : int { KIND_COUPLED = 0, KIND_FLOW = 1, KIND_ADE = 2 };

// Default threads per block of the step kernels.
enum : int { DEFAULT_BLOCK = 128 };

// Everything a step launch needs, independent of dimension and storage type.
struct StepHost {
    int dim, half;
    int dbl;  // FP64 storage and arithmetic (the double-precision instantiation)
    int aq;  // transport velocity set: 5 / 7 (default) or 9 (D2Q9, 2-D)
    int kind, mode;
    Geo geo;
    int bc[3];
    int nblocks;      // out: blocks of the launch (one reduction partial each)
    int grid, block;  // grid.x (blocks along a row) and threads per block
    int idx32;        // every population array has fewer than 2^31 elements: 32-bit offsets
    const void *fsrc;
    void *fdst;
    const void *gsrc;
    void *gdst;
    const void *link;
    void *fld_rho, *fld_u, *fld_c;  // fields in the arithmetic type (FP32, or FP64 when dbl)
    double *partials;
    // parameters in double; the argument block holds them in the arithmetic type
    double omega, omega_c, k_sink, u_scale, rho_out, c_ref;
    double k_half;  // half-saturation concentration of the consumption (0: first order)
    int ade_dirichlet;
    int cut[2];  // the low / high face of the flow axis is a cut (slab decomposition)
    unsigned long long *bounds_err;  // checking builds: the lattice's out-of-range record
    double bb_in[19], gin_dev[9], gout_dev[9];  // per flow / transport direction (at most 19 / 9)
};

// One launch of the batch step kernel over a tile table (coupled steps).
struct BatchHost {
    int dim, half, mode;
    const void *inst;   // device array of per-slot argument blocks, two per slot
    const Tile *tiles;  // device tile table
    const int *ntiles;  // device tile count
    double *partials;   // NSUM per tile
    int parity;
    int grid, block;
};

cudaError_t launch_step_2d_f32(StepHost &h, cudaStream_t s);
cudaError_t launch_step_2d_f16(StepHost &h, cudaStream_t s);
cudaError_t launch_step_3d_f32(StepHost &h, cudaStream_t s);
cudaError_t launch_step_3d_f16(StepHost &h, cudaStream_t s);
// Ghost cells of the buffers h.fdst / h.gdst from the state they hold.
cudaError_t launch_fill_ghosts_2d_f32(const StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_2d_f16(const StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_3d_f32(const StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_3d_f16(const StepHost &h, cudaStream_t s);
cudaError_t launch_step_2d9_f32(StepHost &h, cudaStream_t s);
cudaError_t launch_step_2d9_f16(StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_2d9_f32(const StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_2d9_f16(const StepHost &h, cudaStream_t s);
// The FP64 instantiation (parity reference; single lattices only)
cudaError_t launch_step_2d_f64(StepHost &h, cudaStream_t s);
cudaError_t launch_step_3d_f64(StepHost &h, cudaStream_t s);
cudaError_t launch_step_2d9_f64(StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_2d_f64(const StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_3d_f64(const StepHost &h, cudaStream_t s);
cudaError_t launch_fill_ghosts_2d9_f64(const StepHost &h, cudaStream_t s);

cudaError_t launch_batch_2d_f32(const BatchHost &h, cudaStream_t s);
cudaError_t launch_batch_2d_f16(const BatchHost &h, cudaStream_t s);
cudaError_t launch_batch_3d_f32(const BatchHost &h, cudaStream_t s);
cudaError_t launch_batch_3d_f16(const BatchHost &h, cudaStream_t s);
// The device argument block of a step (StepArgs of the lattice's dimension and storage type)
// written to out (when not null); returns its size in bytes.
size_t step_args_2d_f32(const StepHost &h, void *out);
size_t step_args_2d_f16(const StepHost &h, void *out);
size_t step_args_3d_f32(const StepHost &h, void *out);
size_t step_args_3d_f16(const StepHost &h, void *out);

int batch_occupancy_2d_f32(int block);
int batch_occupancy_2d_f16(int block);
int batch_occupancy_3d_f32(int block);
int batch_occupancy_3d_f16(int block);

inline int batch_occupancy(int dim, int half, int block)
{
    if (dim == 2) return half ? batch_occupancy_2d_f16(block) : batch_occupancy_2d_f32(block);
    return half ? batch_occupancy_3d_f16(block) : batch_occupancy_3d_f32(block);
}

inline cudaError_t launch_batch(const BatchHost &h, cudaStream_t s)
{
    if (h.dim == 2) return h.half ? launch_batch_2d_f16(h, s) : launch_batch_2d_f32(h, s);
    return h.half ? launch_batch_3d_f16(h, s) : launch_batch_3d_f32(h, s);
}

inline size_t step_args(const StepHost &h, void *out)
{
    if (h.dim == 2) return h.half ? step_args_2d_f16(h, out) : step_args_2d_f32(h, out);
    return h.half ? step_args_3d_f16(h, out) : step_args_3d_f32(h, out);
}

inline cudaError_t launch_step(StepHost &h, cudaStream_t s)
{
    if (h.dbl) return h.dim == 3 ? launch_step_3d_f64(h, s) : (h.aq == 9 ? launch_step_2d9_f64(h, s) : launch_step_2d_f64(h, s));
    if (h.dim == 2 && h.aq == 9) return h.half ? launch_step_2d9_f16(h, s) : launch_step_2d9_f32(h, s);
    if (h.dim == 2) return h.half ? launch_step_2d_f16(h, s) : launch_step_2d_f32(h, s);
    return h.half ? launch_step_3d_f16(h, s) : launch_step_3d_f32(h, s);
}

inline cudaError_t launch_fill_ghosts(const StepHost &h, cudaStream_t s)
{
    if (h.dbl)
        return h.dim == 3 ? launch_fill_ghosts_3d_f64(h, s)
                          : (h.aq == 9 ? launch_fill_ghosts_2d9_f64(h, s) : launch_fill_ghosts_2d_f64(h, s));
    if (h.dim == 2 && h.aq == 9) return h.half ? launch_fill_ghosts_2d9_f16(h, s) : launch_fill_ghosts_2d9_f32(h, s);
    if (h.dim == 2) return h.half ? launch_fill_ghosts_2d_f16(h, s) : launch_fill_ghosts_2d_f32(h, s);
    return h.half ? launch_fill_ghosts_3d_f16(h, s) : launch_fill_ghosts_3d_f32(h, s);
}
cudaError_t launch_links(int dim, int aq, const MaskArgs &m, cudaStream_t s);
cudaError_t launch_grow(int dim, const GrowArgs &g, cudaStream_t s);
cudaError_t launch_finalize(const double *partials, int nblocks, double *stage1, double *results,
                            cudaStream_t s);
cudaError_t launch_fields_to_dense(const ConvArgs &a, cudaStream_t s);
cudaError_t launch_pop_convert(const PopArgs &a, cudaStream_t s);

}  // namespace mfc
