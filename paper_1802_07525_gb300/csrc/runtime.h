// Host-side lattice object shared by the single-lattice C ABI (runtime.cu) and the batch engine
// (batch.cu).  Not part of the public interface.
#pragma once

#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mfc.h"
#include "mfc_internal.h"

namespace mfc {

struct GraphEntry {
    int kind, K, fpar, gpar;
    cudaGraphExec_t exec;
};

}  // namespace mfc

struct mfc_lattice {
    mfc_lattice_desc desc;
    mfc_params prm;
    int dim = 2, qf = 9, qa = 5, half = 0;
    int dbl = 0;  // FP64 storage, arithmetic and fields (MFC_FP64)
    int nx = 1, ny = 1, nz = 1;
    mfc::Geo geo;
    long long N = 0;
    size_t st_bytes = 4;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // stream-ordered pool the device buffers come from (batch instances), or null (cudaMalloc)
    cudaMemPool_t pool = nullptr;
    void *f[2] = {nullptr, nullptr};
    void *g[2] = {nullptr, nullptr};
    int fcur = 0, gcur = 0;  // buffer holding the current state (read by the next step)
    void *link = nullptr;
    int link32 = 0;
    uint8_t *cls_cur = nullptr, *cls_tmp = nullptr;
    // fields (rho - 1, u, C - c_ref): FP32, or FP64 in the FP64 instantiation (dbl)
    void *fld_rho = nullptr, *fld_u = nullptr, *fld_c = nullptr;
    double *partials = nullptr;
    double *results_d = nullptr, *results_h = nullptr;
    unsigned long long *counts_d = nullptr, *counts_h = nullptr;
    double *staging = nullptr;
    size_t staging_bytes = 0;
    cudaEvent_t done = nullptr;
    float c_ref = 1.0f;
    int grid = 1, block = mfc::DEFAULT_BLOCK, nblocks = 1, max_blocks = 1;
    int offsets32 = 1;  // plain steps with 32-bit element offsets where the arrays allow

    // checking builds (MFC_CHECK_BOUNDS): the out-of-range record of the step kernels, and the
    // guard regions around every device buffer (allocation base, bytes between the guards)
    unsigned long long *bounds_err = nullptr;
    std::vector<std::pair<char *, size_t>> guards;
    // slab decomposition: the neighbours' classes next to the cut faces (device planes, or null)
    uint8_t *halo_cls[2] = {nullptr, nullptr};
    // agent-based biofilm (allocated by the first mfc_agent_step or mfc_write_biomass)
    double *biomass = nullptr;                // C^bio per node, dense (x fastest)
    unsigned long long *agent_keys = nullptr; // attachment keys per node
    int *agent_list = nullptr;                // nodes above C_max^bio, in increasing order
    int *agent_mark = nullptr;                // position on the current walk's path, or -1
    int *agent_path = nullptr;                // the walk's path
    int agent_path_cap = 0;
    void *agent_state = nullptr;              // selection state and counters

    std::vector<mfc::GraphEntry> graphs;
    long flow_open = 0, ade_open = 0;
    double last_current = 0.0;
    size_t bytes = 0;
    std::string err;
    mfc_status sticky = MFC_OK;
};

namespace mfc {

// Create a lattice like mfc_create_lattice; with a pool, every device buffer is allocated from
// it on the lattice's stream (desc->stream must then be given) and freed back to it.
mfc_status lattice_create(const mfc_lattice_desc *desc, const mfc_params *params, cudaMemPool_t pool,
                          mfc_lattice **out, std::string *why);
// The checks mfc_create_lattice applies to a descriptor and parameters.
mfc_status validate_lattice(const mfc_lattice_desc *desc, const mfc_params *params, std::string *why);
// Elements of the largest population array of a lattice of this descriptor (the larger set's Q
// times the pitched plane): the batch kernel addresses them with 32-bit offsets.
long long lattice_max_elements(const mfc_lattice_desc *desc);
// Step arguments of the lattice for one step of `kind` in `mode` from its current buffers.
void fill_step(const mfc_lattice *L, int kind, int mode, StepHost *h);
// Seconds on the steady clock (the clock of mfc_clock and of the batch time stamps).
double now_s();
// Make the lattice's device current; refuse a lattice with a recorded CUDA error.
mfc_status lattice_enter(mfc_lattice *L);
// Record an error on the lattice (CUDA errors stick) and return s.
mfc_status lattice_fail(mfc_lattice *L, mfc_status s, const std::string &msg);
// Zero-filled device allocation on the lattice's stream (false when it fails); freed with the
// lattice.
bool lattice_alloc(mfc_lattice *L, void **p, size_t bytes);
void lattice_free(mfc_lattice *L, void *p);
// Replace the node classes by the device array dev_cls (N bytes) and rebuild the link masks;
// reset != 0 returns every open node to rest, else a warm start.  Blocks.
mfc_status lattice_apply_classes(mfc_lattice *L, const uint8_t *dev_cls, int reset);
// The fields of the last stepping call as dense doubles (as mfc_read_fields gives them), queued
// on the lattice stream into host buffers (each may be null); the caller waits for the stream.
mfc_status lattice_fields_async(mfc_lattice *L, double *rho, double *u, double *c);
// Free a pooled lattice without waiting for its stream (its frees are stream-ordered).
void lattice_destroy_ordered(mfc_lattice *L);

}  // namespace mfc
