// Batch engine: many steady solves sharing one GPU, with continuous batching (the batch part of
// the C ABI in include/mfc.h).
//
// Requests wait in a first-come-first-served queue and are admitted while an instance slot is
// free and the request's device memory fits the budget.  An admitted request becomes a lattice
// (mfc_lattice) whose buffers come from the batch's stream-ordered memory pool.  All active
// instances of one dimension advance in one launch per step: a fixed grid (resident blocks per
// SM x SMs) walks a tile table listing every row segment of every instance, instance after
// instance (lbm_batch_kernel).  A block is a CUDA graph of K steps (K - 1 plain, one check) per
// group of dimensions present, the per-instance FP64 sums over each instance's tiles, and one
// copy of all instances' sums to pinned host memory.
//
// The host work between blocks overlaps the GPU.  One engine turn, with block b in flight:
//   1. admit queued requests on a side stream (lattice creation, class upload, link masks);
//      they wait outside the tables of block b ("joining");
//   2. wait for block b; free the lattices retired after block b - 1 (their memory is released
//      in stream order, behind block b);
//   3. apply every active instance's stopping test to block b's sums; queue the finished ones'
//      field copies (dense conversion and a copy into pinned staging) on the stream;
//   4. rebuild the tile tables (finished instances out, joining ones in) and launch block b + 1;
//   5. while block b + 1 runs: wait for the copies, hand the fields to the callers' buffers and
//      finish those requests.
// So the GPU idles between blocks only for the stopping test, the table upload and the graph
// launch; a request admitted during block b starts with block b + 1.
//
// Every instance sees exactly the arithmetic it would see alone: its tiles, partial sums and the
// order of their addition depend only on its own shape and the batch's block size, and its
// checks fall every K of its own steps.  K is even, so every instance is back on buffer A at
// every block boundary and one pair of argument blocks (parity 0 and 1) per instance serves
// every block.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/mfc.h"
#include "mfc_internal.h"
#include "runtime.h"

namespace mfc {
namespace {

// Per instance slot, the FP64 sums over the slot's tiles of one group (one block per slot;
// slots of other groups have an empty range and are skipped).
__global__ void __launch_bounds__(256) batch_finalize_kernel(const int2 *ranges, const double *partials,
                                                             double *results)
{
    const int2 r = ranges[blockIdx.x];
    if (r.y <= r.x) return;
    batch_finalize_slot(r, partials, results + (size_t)blockIdx.x * NRESULT);
}

constexpr int NGROUP = 2;  // 2-D and 3-D instances
enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2 };

struct Request {
    long long ticket = 0;
    mfc_lattice_desc desc;
    mfc_params prm;
    std::vector<uint8_t> cls;
    mfc_solve_opts opts;
    double *rho = nullptr, *u = nullptr, *c = nullptr;
    size_t bytes = 0;
    mfc_batch_result res;
    int state = REQ_QUEUED;
};

// Device tables of the instances of one dimension.
struct Group {
    int dim = 2;
    size_t arg_bytes = 0;          // size of one argument block (StepArgs of the group)
    void *inst_d = nullptr;        // 2 * slots argument blocks
    uint8_t *inst_h = nullptr;     // pinned staging of the same
    Tile *tiles_d = nullptr, *tiles_h = nullptr;
    int tile_cap = 0, ntiles = 0;
    int *ntiles_d = nullptr, *ntiles_h = nullptr;
    int2 *ranges_d = nullptr, *ranges_h = nullptr;  // per slot
    double *partials_d = nullptr;  // NSUM per tile
    int grid = 1;
};

enum { SLOT_FREE = 0, SLOT_ACTIVE = 1, SLOT_JOINING = 2, SLOT_RETIRED = 3 };

struct Slot {
    std::shared_ptr<Request> req;  // the request (kept until the lattice is freed)
    mfc_lattice *L = nullptr;
    long steps = 0;
    int state = SLOT_FREE;         // ACTIVE: in the tables of the block in flight; JOINING: admitted
                                   // during a block, active from the next one; RETIRED: finished,
                                   // its lattice freed once the next block is done
    size_t stage = 0;              // retiring: offset of its fields in the pinned staging (doubles)
};

}  // namespace
}  // namespace mfc

using namespace mfc;

struct mfc_batch {
    mfc_batch_opts opts;
    int device = 0, sm_count = 1, half = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    cudaEvent_t done = nullptr, t0 = nullptr, t1 = nullptr;
    cudaEvent_t copies = nullptr;   // the finished instances' field copies of this turn
    cudaStream_t side = nullptr;    // admissions' set-up, overlapping the block in flight
    bool inflight = false;          // a block is queued and its sums not yet applied
    double *stage_h = nullptr;      // pinned staging of finished instances' fields
    size_t stage_cap = 0;           // doubles
    int max_slots = 256;
    int K = 0, block = 0;
    bool tuned = false;
    Group grp[NGROUP];
    double *results_d = nullptr, *results_h = nullptr;
    std::vector<Slot> slots;
    bool tables_dirty = true;
    cudaGraphExec_t graphs[1 << NGROUP] = {};

    // shared with submitting threads (under mu)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<long long, std::shared_ptr<Request>> tickets;
    long long next_ticket = 1;
    size_t used = 0, peak = 0;
    long long submitted = 0, completed = 0, running = 0, blocks = 0, instance_steps = 0;
    std::string err;
    mfc_status sticky = MFC_OK;

    std::atomic<bool> busy{false};  // an engine (mfc_batch_run or the thread) is running
    std::thread thread;
    std::atomic<bool> stop{false};
    bool thread_running = false;
};

namespace {


#define BCK(B, call)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return batch_fail(B, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Record a CUDA failure: the batch stops working and every unfinished request ends with it.
mfc_status batch_fail(mfc_batch *B, const std::string &msg)
{
    std::lock_guard<std::mutex> lock(B->mu);
    B->err = msg;
    B->sticky = MFC_ERR_CUDA;
    return MFC_ERR_CUDA;
}

void finish_locked(mfc_batch *B, const std::shared_ptr<Request> &r, mfc_status st)
{
    r->res.result.status = st;
    r->res.t_done = now_s();
    r->state = REQ_DONE;
    ++B->completed;
    B->cv_done.notify_all();
}

void free_group(Group &g)
{
    cudaFree(g.inst_d);
    cudaFree(g.tiles_d);
    cudaFree(g.ntiles_d);
    cudaFree(g.ranges_d);
    cudaFree(g.partials_d);
    if (g.inst_h) cudaFreeHost(g.inst_h);
    if (g.tiles_h) cudaFreeHost(g.tiles_h);
    if (g.ntiles_h) cudaFreeHost(g.ntiles_h);
    if (g.ranges_h) cudaFreeHost(g.ranges_h);
    g = Group();
}

void drop_graphs(mfc_batch *B)
{
    for (auto &g : B->graphs) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Admit queued requests, first come first served, while a slot is free and the head fits.  Each
// lattice is created and set up on stream `s` (the side stream while a block runs, so that the
// set-up overlaps it), then handed to the batch stream.  With `join`, the new instances wait
// outside the tables of the block in flight and become active with the next one.
mfc_status admit(mfc_batch *B, cudaStream_t s, bool join)
{
    for (;;) {
        std::shared_ptr<Request> r;
        int slot = -1;
        {
            std::lock_guard<std::mutex> lock(B->mu);
            if (B->queue.empty() || B->sticky != MFC_OK) return B->sticky;
            for (int k = 0; k < B->max_slots; ++k)
                if (B->slots[k].state == SLOT_FREE) {
                    slot = k;
                    break;
                }
            if (slot < 0) return MFC_OK;
            r = B->queue.front();
            if (B->used + r->bytes > B->opts.budget_bytes) return MFC_OK;
            B->queue.pop_front();
            B->used += r->bytes;
            B->peak = std::max(B->peak, B->used);
            r->state = REQ_RUNNING;
            ++B->running;
        }
        mfc_lattice_desc d = r->desc;
        d.stream = s;
        mfc_lattice *L = nullptr;
        std::string why;
        mfc_status st = lattice_create(&d, &r->prm, B->pool, &L, &why);
        if (st == MFC_OK) {
            st = mfc_set_geometry(L, r->cls.data(), 1);  // waits for stream s only
            if (st != MFC_OK) {
                why = mfc_last_error(L);
                mfc_destroy_lattice(L);
                L = nullptr;
            }
        }
        std::vector<uint8_t>().swap(r->cls);
        if (st != MFC_OK) {  // the request ends here; the batch carries on unless CUDA failed
            std::lock_guard<std::mutex> lock(B->mu);
            B->used -= r->bytes;
            --B->running;
            finish_locked(B, r, st);
            if (st == MFC_ERR_CUDA) {
                B->err = why;
                B->sticky = MFC_ERR_CUDA;
                return MFC_ERR_CUDA;
            }
            continue;
        }
        L->stream = B->stream;  // its set-up on s is complete: from now on it lives on the batch stream
        r->res.t_admit = now_s();
        Slot &sl = B->slots[slot];
        sl.L = L;
        sl.req = r;
        sl.steps = 0;
        sl.state = join ? SLOT_JOINING : SLOT_ACTIVE;
        B->tables_dirty = true;
    }
}

mfc_status ensure_tiles(mfc_batch *B, Group &g, int need)
{
    if (need <= g.tile_cap) return MFC_OK;
    const int cap = std::max(need, 2 * g.tile_cap);
    BCK(B, cudaStreamSynchronize(B->stream));
    cudaFree(g.tiles_d);
    cudaFree(g.partials_d);
    if (g.tiles_h) cudaFreeHost(g.tiles_h);
    g.tiles_d = nullptr;
    g.partials_d = nullptr;
    g.tiles_h = nullptr;
    g.tile_cap = 0;
    BCK(B, cudaMalloc((void **)&g.tiles_d, (size_t)cap * sizeof(Tile)));
    BCK(B, cudaMalloc((void **)&g.partials_d, (size_t)cap * NSUM * sizeof(double)));
    BCK(B, cudaHostAlloc((void **)&g.tiles_h, (size_t)cap * sizeof(Tile), cudaHostAllocDefault));
    g.tile_cap = cap;
    drop_graphs(B);  // the graphs hold the old table addresses
    return MFC_OK;
}

// Tile tables, ranges and argument blocks of the resident instances, uploaded on the stream.
mfc_status rebuild_tables(mfc_batch *B)
{
    std::vector<Tile> tiles[NGROUP];
    for (int gi = 0; gi < NGROUP; ++gi)
        for (int s = 0; s < B->max_slots; ++s) B->grp[gi].ranges_h[s] = make_int2(0, 0);
    for (int s = 0; s < B->max_slots; ++s) {
        mfc_lattice *L = B->slots[s].L;
        if (!L || B->slots[s].state != SLOT_ACTIVE) continue;
        const int gi = L->dim == 2 ? 0 : 1;
        Group &g = B->grp[gi];
        std::vector<Tile> &t = tiles[gi];
        const int t0 = (int)t.size();
        for (int z = 0; z < L->nz; ++z)
            for (int y = 0; y < L->ny; ++y)
                for (int x0 = 0; x0 < L->nx; x0 += B->block) t.push_back(Tile{s, x0, y, z});
        g.ranges_h[s] = make_int2(t0, (int)t.size());
        StepHost h;
        for (int p = 0; p < 2; ++p) {  // argument blocks of the two buffer parities
            L->fcur = L->gcur = p;
            fill_step(L, KIND_COUPLED, MODE_PLAIN, &h);
            step_args(h, g.inst_h + (size_t)(2 * s + p) * g.arg_bytes);
        }
        L->fcur = L->gcur = 0;
    }
    for (int gi = 0; gi < NGROUP; ++gi) {
        Group &g = B->grp[gi];
        const int n = (int)tiles[gi].size();
        mfc_status st = ensure_tiles(B, g, std::max(n, 1));
        if (st != MFC_OK) return st;
        if (n) memcpy(g.tiles_h, tiles[gi].data(), (size_t)n * sizeof(Tile));
        g.ntiles = n;
        *g.ntiles_h = n;
        if (n) BCK(B, cudaMemcpyAsync(g.tiles_d, g.tiles_h, (size_t)n * sizeof(Tile), cudaMemcpyHostToDevice, B->stream));
        BCK(B, cudaMemcpyAsync(g.ntiles_d, g.ntiles_h, sizeof(int), cudaMemcpyHostToDevice, B->stream));
        BCK(B, cudaMemcpyAsync(g.ranges_d, g.ranges_h, (size_t)B->max_slots * sizeof(int2), cudaMemcpyHostToDevice,
                               B->stream));
        BCK(B, cudaMemcpyAsync(g.inst_d, g.inst_h, (size_t)2 * B->max_slots * g.arg_bytes, cudaMemcpyHostToDevice,
                               B->stream));
    }
    B->tables_dirty = false;
    return MFC_OK;
}

BatchHost batch_host(const mfc_batch *B, const Group &g, int mode, int parity)
{
    BatchHost h;
    h.dim = g.dim;
    h.half = B->half;
    h.mode = mode;
    h.inst = g.inst_d;
    h.tiles = g.tiles_d;
    h.ntiles = g.ntiles_d;
    h.partials = g.partials_d;
    h.parity = parity;
    h.grid = g.grid;
    h.block = B->block;
    return h;
}

mfc_status set_block(mfc_batch *B, int block)
{
    B->block = block;
    for (int gi = 0; gi < NGROUP; ++gi)
        B->grp[gi].grid = B->sm_count * batch_occupancy(B->grp[gi].dim, B->half, block);
    drop_graphs(B);
    B->tables_dirty = true;
    return rebuild_tables(B);
}

// Pick the block size by timing plain steps of the resident instances, and K (when not given)
// from the measured step time and check overhead.  The timed steps read buffer A and write
// buffer B of every instance; the next real step rewrites everything of B that is read later,
// so tuning changes no result.
mfc_status autotune(mfc_batch *B)
{
    std::vector<int> cand;
    if (B->opts.block) cand.push_back(B->opts.block);
    else cand = {64, 128, 256};
    double best = 1e30;
    int best_block = cand[0];
    for (int blk : cand) {
        mfc_status st = set_block(B, blk);
        if (st != MFC_OK) return st;
        const int reps = 5;
        for (int r = -2; r < reps; ++r) {
            if (r == 0) BCK(B, cudaEventRecord(B->t0, B->stream));
            for (int gi = 0; gi < NGROUP; ++gi)
                if (B->grp[gi].ntiles) BCK(B, launch_batch(batch_host(B, B->grp[gi], MODE_PLAIN, 0), B->stream));
        }
        BCK(B, cudaEventRecord(B->t1, B->stream));
        BCK(B, cudaEventSynchronize(B->t1));
        float ms = 0.f;
        BCK(B, cudaEventElapsedTime(&ms, B->t0, B->t1));
        const double t = ms * 1e-3 / reps;
        if (t < best) {
            best = t;
            best_block = blk;
        }
    }
    if (B->block != best_block) {
        mfc_status st = set_block(B, best_block);
        if (st != MFC_OK) return st;
    }
    if (B->K == 0) {
        // check overhead: the sums of every group, the copy to the host and the host's wait,
        // plus the check step's extra traffic (about 40% of a plain step)
        const double h0 = now_s();
        for (int gi = 0; gi < NGROUP; ++gi)
            if (B->grp[gi].ntiles)
                batch_finalize_kernel<<<B->max_slots, 256, 0, B->stream>>>(B->grp[gi].ranges_d, B->grp[gi].partials_d,
                                                                           B->results_d);
        BCK(B, cudaGetLastError());
        BCK(B, cudaMemcpyAsync(B->results_h, B->results_d, (size_t)B->max_slots * NRESULT * sizeof(double),
                               cudaMemcpyDeviceToHost, B->stream));
        BCK(B, cudaEventRecord(B->done, B->stream));
        BCK(B, cudaEventSynchronize(B->done));
        const double t_o = (now_s() - h0) + 0.4 * best;
        // expected steps per solve: the first resident request's cap, at most 20000
        double S = 20000.0;
        for (auto &sl : B->slots)
            if (sl.state == SLOT_ACTIVE && sl.req->opts.max_steps > 0)
                S = std::min(S, (double)sl.req->opts.max_steps);
        // blocks cost t_o each and a converged solve overshoots by K/2 steps on average:
        // S t_o / K + K t_step / 2 is least at K = sqrt(2 S t_o / t_step)
        double k = sqrt(2.0 * S * t_o / std::max(best, 1e-9));
        int K = (int)std::min(2000.0, std::max(20.0, k));
        B->K = K + (K & 1);
        drop_graphs(B);
    }
    B->tuned = true;
    return MFC_OK;
}

// The graph of one block for the groups in `mask`.
mfc_status graph_for(mfc_batch *B, int mask, cudaGraphExec_t *out)
{
    if (B->graphs[mask]) {
        *out = B->graphs[mask];
        return MFC_OK;
    }
    BCK(B, cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < B->K && e == cudaSuccess; ++s) {
        const int mode = s == B->K - 1 ? MODE_CHECK : MODE_PLAIN;
        for (int gi = 0; gi < NGROUP && e == cudaSuccess; ++gi)
            if (mask & (1 << gi)) e = launch_batch(batch_host(B, B->grp[gi], mode, s & 1), B->stream);
    }
    for (int gi = 0; gi < NGROUP && e == cudaSuccess; ++gi)
        if (mask & (1 << gi)) {
            batch_finalize_kernel<<<B->max_slots, 256, 0, B->stream>>>(B->grp[gi].ranges_d, B->grp[gi].partials_d,
                                                                       B->results_d);
            e = cudaGetLastError();
        }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->results_h, B->results_d, (size_t)B->max_slots * NRESULT * sizeof(double),
                            cudaMemcpyDeviceToHost, B->stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(B->stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return batch_fail(B, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return batch_fail(B, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    B->graphs[mask] = exec;
    *out = exec;
    return MFC_OK;
}

// Pinned staging for `need` doubles of finished instances' fields (its previous contents have
// been handed out already).
mfc_status ensure_stage(mfc_batch *B, size_t need)
{
    if (need <= B->stage_cap) return MFC_OK;
    const size_t cap = std::max(need, 2 * B->stage_cap);
    if (B->stage_h) cudaFreeHost(B->stage_h);
    B->stage_h = nullptr;
    B->stage_cap = 0;
    BCK(B, cudaHostAlloc((void **)&B->stage_h, cap * sizeof(double), cudaHostAllocDefault));
    B->stage_cap = cap;
    return MFC_OK;
}

// Free the lattices retired after the previous block (the stream is idle or runs a block that
// does not use them: their frees are stream-ordered) and return their memory to the budget.
void free_retired(mfc_batch *B)
{
    for (auto &sl : B->slots) {
        if (sl.state != SLOT_RETIRED) continue;
        lattice_destroy_ordered(sl.L);
        sl.L = nullptr;
        sl.state = SLOT_FREE;
        {
            std::lock_guard<std::mutex> lock(B->mu);
            B->used -= sl.req->bytes;
        }
        sl.req.reset();
    }
}

// Apply every active instance's stopping test to the sums of the block just run.  The finished
// ones leave the tables; the copies of their fields into the pinned staging are queued on the
// stream (ahead of the next block) and marked by B->copies.  *finished counts them.
mfc_status retire_decide(mfc_batch *B, int *finished)
{
    *finished = 0;
    const double now = now_s();
    size_t need = 0;
    std::vector<int> done;
    for (int s = 0; s < B->max_slots; ++s) {
        Slot &sl = B->slots[s];
        if (sl.state != SLOT_ACTIVE) continue;
        sl.steps += B->K;
        const double *r = B->results_h + (size_t)s * NRESULT;
        const double rf = r[RES_FLOW] / B->K, ra = r[RES_ADE] / B->K;
        Request &q = *sl.req;
        mfc_solve_result &res = q.res.result;
        res.steps_flow = res.steps_ade = sl.steps;
        res.res_flow = rf;
        res.res_ade = ra;
        res.current = r[SUM_CURRENT];
        res.mass = r[SUM_MASS];
        res.substrate = r[SUM_C];
        mfc_status st;
        if (r[SUM_BAD] > 0.0 || !isfinite(r[SUM_MASS]) || !isfinite(r[SUM_C]) || isnan(rf) || isnan(ra))
            st = MFC_ERR_NONFINITE;
        else if (r[SUM_FAST] > 0.0)
            st = MFC_ERR_UNSTABLE;
        else if (rf < q.opts.tol_flow && ra < q.opts.tol_ade)
            st = MFC_OK;
        else if (sl.steps >= q.opts.max_steps)
            st = MFC_NOT_CONVERGED;
        else if (q.opts.timeout_s > 0.0 && now - q.res.t_admit > q.opts.timeout_s)
            st = MFC_ERR_TIMEOUT;
        else
            continue;
        res.status = st;
        sl.L->last_current = r[SUM_CURRENT];
        sl.state = SLOT_RETIRED;
        sl.stage = need;
        if (q.rho || q.u || q.c) need += (size_t)(2 + sl.L->dim) * (size_t)sl.L->N;
        done.push_back(s);
        B->tables_dirty = true;
    }
    *finished = (int)done.size();
    if (done.empty()) return MFC_OK;
    mfc_status st = ensure_stage(B, need);
    if (st != MFC_OK) return st;
    for (int s : done) {
        Slot &sl = B->slots[s];
        Request &q = *sl.req;
        if (!(q.rho || q.u || q.c)) continue;
        const size_t N = (size_t)sl.L->N;
        double *base = B->stage_h + sl.stage;
        st = lattice_fields_async(sl.L, q.rho ? base : nullptr, q.u ? base + N : nullptr,
                                  q.c ? base + (1 + sl.L->dim) * N : nullptr);
        if (st != MFC_OK) return batch_fail(B, "reading the fields of a finished instance failed");
    }
    BCK(B, cudaEventRecord(B->copies, B->stream));
    return MFC_OK;
}

// Hand the finished instances' fields to their callers (after their copies) and finish the
// requests.  Their lattices stay allocated until the block now in flight is done.
mfc_status retire_complete(mfc_batch *B)
{
    BCK(B, cudaEventSynchronize(B->copies));
    for (auto &sl : B->slots) {
        if (sl.state != SLOT_RETIRED || sl.req->state == REQ_DONE) continue;
        Request &q = *sl.req;
        const size_t N = (size_t)sl.L->N;
        const double *base = B->stage_h + sl.stage;
        if (q.rho) memcpy(q.rho, base, N * sizeof(double));
        if (q.u) memcpy(q.u, base + N, (size_t)sl.L->dim * N * sizeof(double));
        if (q.c) memcpy(q.c, base + (1 + sl.L->dim) * N, N * sizeof(double));
        std::lock_guard<std::mutex> lock(B->mu);
        --B->running;
        finish_locked(B, sl.req, (mfc_status)q.res.result.status);
    }
    return MFC_OK;
}

int active_mask(const mfc_batch *B, long long *n_active)
{
    int mask = 0;
    long long n = 0;
    for (auto &sl : B->slots)
        if (sl.state == SLOT_ACTIVE) {
            mask |= 1 << (sl.L->dim == 2 ? 0 : 1);
            ++n;
        }
    if (n_active) *n_active = n;
    return mask;
}

// Queue one block of every active instance.
mfc_status launch_block(mfc_batch *B, int mask, long long n_active)
{
    if (!B->tuned) {
        mfc_status st = autotune(B);
        if (st != MFC_OK) return st;
    }
    if (B->tables_dirty) {
        mfc_status st = rebuild_tables(B);
        if (st != MFC_OK) return st;
    }
    cudaGraphExec_t exec;
    mfc_status st = graph_for(B, mask, &exec);
    if (st != MFC_OK) return st;
    BCK(B, cudaGraphLaunch(exec, B->stream));
    BCK(B, cudaEventRecord(B->done, B->stream));
    B->inflight = true;
    std::lock_guard<std::mutex> lock(B->mu);
    ++B->blocks;
    B->instance_steps += n_active * B->K;
    return MFC_OK;
}

// One engine turn (see the file comment).  *worked = false when nothing was in flight, active or
// joining, and nothing could be admitted.
mfc_status engine_turn(mfc_batch *B, bool *worked)
{
    *worked = false;
    mfc_status st;
    if (!B->inflight) {
        // nothing runs: free what retired, admit straight onto the batch stream, start a block
        BCK(B, cudaStreamSynchronize(B->stream));
        free_retired(B);
        st = admit(B, B->stream, false);
        if (st != MFC_OK) return st;
        for (auto &sl : B->slots)
            if (sl.state == SLOT_JOINING) {
                sl.state = SLOT_ACTIVE;
                B->tables_dirty = true;
            }
        long long n = 0;
        const int mask = active_mask(B, &n);
        if (!mask) return MFC_OK;
        *worked = true;
        return launch_block(B, mask, n);
    }
    *worked = true;
    // 1. admissions overlap the block in flight
    st = admit(B, B->side, true);
    if (st != MFC_OK) return st;
    // 2. the block's sums
    BCK(B, cudaEventSynchronize(B->done));
    B->inflight = false;
    free_retired(B);
    // 3. stopping tests; the finished instances' copies go ahead of the next block
    int finished = 0;
    st = retire_decide(B, &finished);
    if (st != MFC_OK) return st;
    // 4. the next block: joining instances in, finished ones out
    for (auto &sl : B->slots)
        if (sl.state == SLOT_JOINING) {
            sl.state = SLOT_ACTIVE;
            B->tables_dirty = true;
        }
    long long n = 0;
    const int mask = active_mask(B, &n);
    if (mask) {
        st = launch_block(B, mask, n);
        if (st != MFC_OK) return st;
    }
    // 5. results of the finished instances, while the next block runs
    if (finished) return retire_complete(B);
    return MFC_OK;
}

// After a CUDA failure: every unfinished request ends with it.
void fail_all(mfc_batch *B)
{
    cudaStreamSynchronize(B->stream);
    cudaGetLastError();
    B->inflight = false;
    for (auto &sl : B->slots) {
        if (!sl.L) continue;
        lattice_destroy_ordered(sl.L);
        sl.L = nullptr;
        std::lock_guard<std::mutex> lock(B->mu);
        B->used -= sl.req->bytes;
        if (sl.req->state != REQ_DONE) {
            --B->running;
            finish_locked(B, sl.req, MFC_ERR_CUDA);
        }
        sl.req.reset();
        sl.state = SLOT_FREE;
    }
    std::lock_guard<std::mutex> lock(B->mu);
    while (!B->queue.empty()) {
        finish_locked(B, B->queue.front(), MFC_ERR_CUDA);
        B->queue.pop_front();
    }
}

void engine_thread(mfc_batch *B)
{
    cudaSetDevice(B->device);
    while (!B->stop.load()) {
        bool worked = false;
        if (engine_turn(B, &worked) != MFC_OK) {
            fail_all(B);
            return;
        }
        if (!worked) {
            std::unique_lock<std::mutex> lock(B->mu);
            B->cv_work.wait_for(lock, std::chrono::milliseconds(50),
                                [&] { return B->stop.load() || !B->queue.empty(); });
        }
    }
}

mfc_status copy_result(mfc_batch *B, long long ticket, mfc_batch_result *out, std::unique_lock<std::mutex> &lock,
                       double timeout_s)
{
    auto it = B->tickets.find(ticket);
    if (it == B->tickets.end()) return MFC_ERR_ARG;
    std::shared_ptr<Request> r = it->second;
    if (r->state != REQ_DONE && timeout_s != 0.0) {
        auto pred = [&] { return r->state == REQ_DONE; };
        if (timeout_s < 0.0) B->cv_done.wait(lock, pred);
        else B->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), pred);
    }
    if (r->state != REQ_DONE) return MFC_PENDING;
    if (out) *out = r->res;
    B->tickets.erase(ticket);
    return (mfc_status)r->res.result.status;
}

}  // namespace

extern "C" {

MFC_API double mfc_clock(void) { return now_s(); }

MFC_API mfc_status mfc_batch_create(const mfc_batch_opts *opts, mfc_batch **out)
{
    if (!opts || !out) return MFC_ERR_ARG;
    *out = nullptr;
    if (opts->precision != MFC_FP32 && opts->precision != MFC_FP16_DEV) return MFC_ERR_ARG;
    if (opts->block != 0 && opts->block != 64 && opts->block != 128 && opts->block != 256) return MFC_ERR_ARG;
    if (opts->check_every < 0 || opts->max_instances < 0 || opts->max_instances > 4096) return MFC_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return MFC_ERR_CUDA;
    }
    mfc_batch *B = new (std::nothrow) mfc_batch();
    if (!B) return MFC_ERR_OOM;
    B->opts = *opts;
    B->half = opts->precision == MFC_FP16_DEV;
    B->max_slots = opts->max_instances ? opts->max_instances : 256;
    B->K = opts->check_every ? opts->check_every + (opts->check_every & 1) : 0;
    B->block = opts->block ? opts->block : DEFAULT_BLOCK;
    B->slots.resize(B->max_slots);
    cudaError_t e = cudaGetDevice(&B->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, B->device);
    if (e == cudaSuccess && !opts->budget_bytes) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        B->opts.budget_bytes = (size_t)(0.9 * (double)fr);
    }
    if (e == cudaSuccess) {
        if (opts->stream) {
            B->stream = (cudaStream_t)opts->stream;
        } else {
            e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
            B->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = B->device;
        e = cudaMemPoolCreate(&B->pool, &props);
        if (e == cudaSuccess) {  // keep freed memory for the next instances
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(B->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->done, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->copies, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&B->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&B->t1);
    if (e == cudaSuccess) e = cudaMalloc((void **)&B->results_d, (size_t)B->max_slots * NRESULT * sizeof(double));
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&B->results_h, (size_t)B->max_slots * NRESULT * sizeof(double), cudaHostAllocDefault);
    for (int gi = 0; gi < NGROUP && e == cudaSuccess; ++gi) {
        Group &g = B->grp[gi];
        g.dim = gi == 0 ? 2 : 3;
        StepHost h;
        memset(&h, 0, sizeof h);
        h.dim = g.dim;
        h.half = B->half;
        // the kernel indexes the blocks as an array of StepArgs: the stride is exactly its size
        g.arg_bytes = step_args(h, nullptr);
        const size_t ib = (size_t)2 * B->max_slots * g.arg_bytes;
        e = cudaMalloc(&g.inst_d, ib);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&g.inst_h, ib, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g.ntiles_d, sizeof(int));
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&g.ntiles_h, sizeof(int), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc((void **)&g.ranges_d, (size_t)B->max_slots * sizeof(int2));
        if (e == cudaSuccess)
            e = cudaHostAlloc((void **)&g.ranges_h, (size_t)B->max_slots * sizeof(int2), cudaHostAllocDefault);
        if (e == cudaSuccess) memset(g.inst_h, 0, ib);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        mfc_batch_destroy(B);
        return e == cudaErrorMemoryAllocation ? MFC_ERR_OOM : MFC_ERR_CUDA;
    }
    *out = B;
    return MFC_OK;
}

MFC_API mfc_status mfc_batch_destroy(mfc_batch *B)
{
    if (!B) return MFC_ERR_ARG;
    mfc_batch_stop(B);
    {
        if (B->stream) cudaStreamSynchronize(B->stream);  // a block may still be in flight
        if (B->side) cudaStreamSynchronize(B->side);
        for (auto &sl : B->slots)
            if (sl.L) {
                mfc_destroy_lattice(sl.L);
                sl.L = nullptr;
            }
        if (B->stream) cudaStreamSynchronize(B->stream);
        drop_graphs(B);
        for (auto &g : B->grp) free_group(g);
        cudaFree(B->results_d);
        if (B->results_h) cudaFreeHost(B->results_h);
        if (B->done) cudaEventDestroy(B->done);
        if (B->copies) cudaEventDestroy(B->copies);
        if (B->side) cudaStreamDestroy(B->side);
        if (B->stage_h) cudaFreeHost(B->stage_h);
        if (B->t0) cudaEventDestroy(B->t0);
        if (B->t1) cudaEventDestroy(B->t1);
        if (B->pool) cudaMemPoolDestroy(B->pool);
        if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    }
    delete B;
    return MFC_OK;
}

MFC_API mfc_status mfc_batch_submit(mfc_batch *B, const mfc_lattice_desc *desc, const mfc_params *params,
                                    const uint8_t *node_class, const mfc_solve_opts *opts, double *rho,
                                    double *u, double *c, long long *ticket)
{
    if (!B || !desc || !params || !node_class || !opts || !ticket) return MFC_ERR_ARG;
    std::string why;
    mfc_lattice_desc d = *desc;
    d.stream = nullptr;
    if (validate_lattice(&d, params, &why) != MFC_OK) return MFC_ERR_ARG;
    if (d.precision != B->opts.precision) return MFC_ERR_ARG;
    if (d.ade_q == 9) return MFC_ERR_ARG;  // batches run the default transport sets
    if (d.cut[0] || d.cut[1]) return MFC_ERR_ARG;  // whole lattices only
    if (lattice_max_elements(&d) >= (1ll << 31)) return MFC_ERR_ARG;  // 32-bit element offsets
    if (opts->mode != MFC_CONCURRENT || opts->max_steps < 0 || !(opts->tol_flow >= 0.0) ||
        !(opts->tol_ade >= 0.0))
        return MFC_ERR_ARG;
    const long long N = (long long)d.nx * d.ny * (d.dim == 2 ? 1 : d.nz);
    for (long long q = 0; q < N; ++q)
        if (node_class[q] > 7) return MFC_ERR_ARG;
    auto r = std::make_shared<Request>();
    r->desc = d;
    r->prm = *params;
    r->opts = *opts;
    r->rho = rho;
    r->u = u;
    r->c = c;
    // the lattice, the read-back staging, and the pool's allocation granularity
    r->bytes = mfc_lattice_bytes(&d) + ((rho || u || c) ? (size_t)(2 + d.dim) * N * sizeof(double) : 0) +
               (size_t)16 * (2u << 20);
    if (r->bytes > B->opts.budget_bytes) return MFC_ERR_OOM_BUDGET;
    r->cls.assign(node_class, node_class + N);
    memset(&r->res, 0, sizeof r->res);
    r->res.t_submit = now_s();
    r->res.result.status = MFC_PENDING;
    {
        std::lock_guard<std::mutex> lock(B->mu);
        if (B->sticky != MFC_OK) return B->sticky;
        r->ticket = B->next_ticket++;
        B->tickets[r->ticket] = r;
        B->queue.push_back(r);
        ++B->submitted;
        *ticket = r->ticket;
    }
    B->cv_work.notify_all();
    return MFC_OK;
}

MFC_API mfc_status mfc_batch_poll(mfc_batch *B, long long ticket, mfc_batch_result *out)
{
    if (!B) return MFC_ERR_ARG;
    std::unique_lock<std::mutex> lock(B->mu);
    return copy_result(B, ticket, out, lock, 0.0);
}

MFC_API mfc_status mfc_batch_wait(mfc_batch *B, long long ticket, double timeout_s, mfc_batch_result *out)
{
    if (!B) return MFC_ERR_ARG;
    std::unique_lock<std::mutex> lock(B->mu);
    return copy_result(B, ticket, out, lock, timeout_s);
}

MFC_API mfc_status mfc_batch_run(mfc_batch *B)
{
    if (!B) return MFC_ERR_ARG;
    bool idle = false;
    if (!B->busy.compare_exchange_strong(idle, true)) return MFC_ERR_STATE;  // an engine is running
    cudaSetDevice(B->device);
    mfc_status st = MFC_OK;
    for (;;) {
        bool worked = false;
        st = engine_turn(B, &worked);
        if (st != MFC_OK) {
            fail_all(B);
            break;
        }
        if (!worked) {
            std::lock_guard<std::mutex> lock(B->mu);
            if (B->queue.empty()) break;
        }
    }
    B->busy.store(false);
    return st;
}

MFC_API mfc_status mfc_batch_start(mfc_batch *B)
{
    if (!B) return MFC_ERR_ARG;
    if (B->thread_running) return MFC_OK;
    bool idle = false;
    if (!B->busy.compare_exchange_strong(idle, true)) return MFC_ERR_STATE;  // mfc_batch_run is running
    B->stop.store(false);
    B->thread_running = true;
    B->thread = std::thread([B] {
        engine_thread(B);
        B->busy.store(false);
    });
    return MFC_OK;
}

MFC_API mfc_status mfc_batch_stop(mfc_batch *B)
{
    if (!B) return MFC_ERR_ARG;
    if (!B->thread_running) return MFC_OK;
    B->stop.store(true);
    B->cv_work.notify_all();
    if (B->thread.joinable()) B->thread.join();
    B->thread_running = false;
    return MFC_OK;
}

MFC_API mfc_status mfc_batch_get_stats(mfc_batch *B, mfc_batch_stats *out)
{
    if (!B || !out) return MFC_ERR_ARG;
    std::lock_guard<std::mutex> lock(B->mu);
    out->submitted = B->submitted;
    out->completed = B->completed;
    out->running = B->running;
    out->queued = (long long)B->queue.size();
    out->blocks = B->blocks;
    out->instance_steps = B->instance_steps;
    out->bytes_in_use = B->used;
    out->bytes_peak = B->peak;
    out->budget_bytes = B->opts.budget_bytes;
    out->check_every = B->K;
    out->block = B->block;
    out->grid = B->grp[0].grid;
    return B->sticky;
}

MFC_API const char *mfc_batch_last_error(mfc_batch *B) { return B ? B->err.c_str() : ""; }

}  // extern "C"
