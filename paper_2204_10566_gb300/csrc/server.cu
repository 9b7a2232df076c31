// Request server: continuous batching of many lattices on one GPU.
//
// Requests (flag field, flow parameters, step count, storage precision) are
// queued by lbm_server_submit; host worker threads build each request's
// sparse index while the GPU is busy.  lbm_server_tick admits ready requests
// into resident slots by exact device footprint against the budget, then
// advances every resident lattice by up to steps_per_tick steps with one
// captured CUDA graph: per step, one persistent multi-lattice fluid launch
// and one boundary launch per precision group.  The blocks of those launches
// walk a tile list that spans all resident lattices (a tile is one block's
// worth of chunks of one lattice); the lattice of a tile is found by binary
// search in a per-tick table that the graph copies to the device first.  The
// table changes every tick, the graph never does.  Each cell is updated by
// the same device code as lbm_step, so a lattice's result does not depend on
// what else is resident.
#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lbm_device.cuh"

namespace lbm {

// FP16S scale of a descriptor (api.cu): 0 selects the default 4096, any
// other value must be a positive power of two; returns 0 when invalid.
float resolve_fp16_scale(float s);

// A context's step arguments in the chunk kernel's view (api.cu): every
// chunk and every inlet/outlet node, whichever fluid kernel its own steps run.
void ctx_chunk_step_args(lbm_ctx *c, StepArgs *out);

constexpr int MAX_SLOTS = LBM_SERVER_MAX_SLOTS;
constexpr int NGROUPS = 2;  // 0: FP32, 1: FP16S

struct alignas(16) DomainEntry {
    StepArgs a;        // state at the start of the tick: fin is the current buffer
    int64_t t_base;    // steps done before the tick
    int32_t steps;     // steps this lattice takes in the tick
    int32_t tile_begin, btile_begin, pad;
};

struct alignas(16) GroupTable {
    int32_t n_domains, n_tiles, n_btiles, pad;
    DomainEntry d[MAX_SLOTS];
};

// Lattice of a tile: the last entry whose first tile is <= tile.
template <bool BND>
__device__ __forceinline__ int find_domain(const GroupTable *tab, int tile) {
    int lo = 0, hi = tab->n_domains - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int begin = BND ? tab->d[mid].btile_begin : tab->d[mid].tile_begin;
        if (begin <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Step k of the tick for the tile's lattice: copy its arguments to shared
// memory, swap the buffers on odd steps, set the step number (inlet noise).
// The lattice's last step of the tick is its health check: every cell then
// computes its non-finite flag (STEP_REDUCE), and a.status points at the
// lattice's word of the server's health-flag array.
__device__ __forceinline__ bool load_domain(const DomainEntry &e, int k, StepArgs &sa) {
    if (k >= e.steps) return false;
    for (int w = threadIdx.x; w < (int)(sizeof(StepArgs) / 16); w += blockDim.x)
        reinterpret_cast<int4 *>(&sa)[w] = reinterpret_cast<const int4 *>(&e.a)[w];
    __syncthreads();
    if (threadIdx.x == 0) {
        if (k & 1) {
            const void *t = sa.fin;
            sa.fin = sa.fout;
            sa.fout = const_cast<void *>(t);
        }
        sa.t_new = e.t_base + k + 1;
        sa.flags = k == e.steps - 1 ? STEP_REDUCE : 0;
    }
    __syncthreads();
    return true;
}

// Health check of a tile on its lattice's check step: one atomic per warp
// that saw a non-finite density or velocity (hv[5], set by record_cell).
__device__ __forceinline__ void flag_non_finite(const StepArgs &sa, const double (&hv)[6]) {
    if (!(sa.flags & STEP_REDUCE)) return;  // uniform over the block
    if (__any_sync(0xffffffffu, hv[5] != 0.0) && (threadIdx.x & 31) == 0) atomicOr(sa.status, 1u);
}

template <int P>
__global__ void __launch_bounds__(STEP_THREADS, LBM_STEP_MIN_BLOCKS) k_multi_fluid(const GroupTable *tab, int k) {
    __shared__ StepArgs sa;
    __shared__ int s_dom;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    const int ntiles = tab->n_tiles;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();  // the previous tile is done with sa
        if (threadIdx.x == 0) s_dom = find_domain<false>(tab, tile);
        __syncthreads();
        const DomainEntry &e = tab->d[s_dom];
        if (!load_domain(e, k, sa)) continue;  // uniform over the block
        const int chunk = (tile - e.tile_begin) * (STEP_THREADS / CHUNK) + threadIdx.x / CHUNK;
        hv[5] = 0.0;
        if (chunk < sa.nchunks) {
            if (sa.row_axis == 2)  // uniform over the block
                fluid_cell<P, true, false, 2>(sa, chunk, threadIdx.x % CHUNK, hv);
            else
                fluid_cell<P, true, false, 0>(sa, chunk, threadIdx.x % CHUNK, hv);
        }
        flag_non_finite(sa, hv);
    }
}

template <int P>
__global__ void __launch_bounds__(STEP_THREADS) k_multi_boundary(const GroupTable *tab, int k) {
    __shared__ StepArgs sa;
    __shared__ int s_dom;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    const int ntiles = tab->n_btiles;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) s_dom = find_domain<true>(tab, tile);
        __syncthreads();
        const DomainEntry &e = tab->d[s_dom];
        if (!load_domain(e, k, sa)) continue;
        const int node = (tile - e.btile_begin) * STEP_THREADS + threadIdx.x;
        hv[5] = 0.0;
        if (node < sa.nbnodes) {
            if (sa.row_axis == 2)
                boundary_node<P, true, false, 2>(sa, node, hv);
            else
                boundary_node<P, true, false, 0>(sa, node, hv);
        }
        flag_non_finite(sa, hv);
    }
}

}  // namespace lbm

using namespace lbm;

namespace {

struct Request {
    int64_t id = 0;
    lbm_request req{};
    std::vector<uint8_t> flags;
    int state = LBM_REQ_QUEUED;
    lbm_status fail_status = LBM_OK;  // why a FAILED request failed
    int64_t steps_done = 0;
    bool cancel = false;
    // built by a worker thread (guarded by the server mutex)
    bool index_ready = false;
    std::string index_error;
    HostIndex idx;
    int64_t footprint = 0;
    int64_t n_active = -1;
    // resident state
    lbm_ctx *ctx = nullptr;
    int group = 0;
    // result
    std::vector<double> rho, u;
};

int storage_size(int precision) { return precision == LBM_FP32 ? 4 : 2; }

}  // namespace

struct lbm_server {
    lbm_server_desc desc{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::deque<int64_t> queue;      // submitted, not yet admitted (submission order)
    std::vector<int64_t> resident;  // admitted, running
    int64_t next_id = 1;
    int64_t in_use = 0, peak = 0;
    double cell_updates = 0, ticks = 0, graph_launches = 0, graph_captures = 0, finished = 0;
    // worker threads building indexes
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> build_queue;
    bool stop = false;
    // device tables and the tick graph
    GroupTable *h_tab[NGROUPS] = {nullptr, nullptr};
    GroupTable *d_tab[NGROUPS] = {nullptr, nullptr};
    // health flags, one word per (group, domain): cleared at the start of
    // every tick, raised by the check step, copied back at its end
    uint32_t *d_flags = nullptr, *h_flags = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid_fluid[NGROUPS] = {0, 0}, grid_bnd[NGROUPS] = {0, 0};
};

namespace {

lbm_status sfail(lbm_server *s, lbm_status st, const std::string &m) {
    if (s) s->err = m;
    return st;
}

// Device bytes a request holds while resident: the context's buffers plus
// the readback staging of its moments.
int64_t request_footprint(const lbm_request &q, const HostIndex &idx) {
    lbm_desc d{};
    d.nx = q.nx;
    d.ny = q.ny;
    d.nz = q.nz;
    d.periodic = q.periodic;
    d.precision = q.precision;
    return ctx_footprint(d, idx) + idx.n_active * 32;
}

// The checks of lbm_server_submit that need no index (host only).  *active
// receives the request's active cell count.
lbm_status check_request(const lbm_request *q, int64_t budget_bytes, int64_t *active, const char **why) {
    *active = 0;
    auto bad = [why](lbm_status st, const char *m) {
        *why = m;
        return st;
    };
    if (!q || !q->flags) return bad(LBM_ERR_ARG, "NULL request or flags");
    if (q->precision != LBM_FP32 && q->precision != LBM_FP16S)
        return bad(LBM_ERR_ARG, "the server runs FP32 and FP16S lattices");
    if (q->steps < 1 || q->nx < 1 || q->ny < 1 || q->nz < 1 || (q->periodic & ~7))
        return bad(LBM_ERR_ARG, "bad lattice size, periodicity or step count");
    const lbm_params &p = q->params;
    if (p.omega3 != 1.0 || p.omega4 != 1.0 || p.omega5 != 1.0 || p.omega6 != 1.0)
        return bad(LBM_ERR_ARG, "the server runs the default ghost rates only");
    if (resolve_fp16_scale(q->fp16_scale) == 0.0f)
        return bad(LBM_ERR_ARG, "the FP16 scale must be 0 (default) or a power of two");
    if (lbm_params_check(&p, nullptr, nullptr, why) != LBM_OK) return LBM_ERR_ARG;  // lbm_set_params' checks
    const int64_t ncell = (int64_t)q->nx * q->ny * q->nz;
    int64_t n = 0;
    for (int64_t b = 0; b < ncell; ++b) n += q->flags[b] != LBM_SOLID;
    *active = n;
    // every active cell has a slot: a lattice this large can never get 32-bit offsets
    if (n > MAX_SLOTS_32)
        return bad(LBM_ERR_ARG, "the lattice has more active cells than the server's 32-bit population "
                                "offsets address (2^32 / 27 slots); run it with lbm_step");
    if (2 * 27 * n * storage_size(q->precision) > budget_bytes)
        return bad(LBM_ERR_OOM, "the lattice can never fit the server's memory budget");
    *why = "";
    return LBM_OK;
}

void worker_loop(lbm_server *s) {
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->build_queue.empty(); });
            if (s->stop) return;
            r = s->build_queue.front();
            s->build_queue.pop_front();
        }
        const TraceRange trace("lbm_server: index build");
        HostIndex idx;
        const lbm_request &q = r->req;
        // the multi-lattice kernels address populations with 32-bit offsets
        std::string e = build_index(r->flags.data(), q.nx, q.ny, q.nz, q.periodic, idx, MAX_SLOTS_32);
        const int64_t fp = e.empty() ? request_footprint(q, idx) : 0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            r->index_error = e;
            r->footprint = fp;
            r->n_active = e.empty() ? idx.n_active : 0;
            r->idx = std::move(idx);
            r->index_ready = true;
        }
    }
}

template <int P>
void occupancy_grids(int sms, int &gf, int &gb) {
    int nf = 0, nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nf, k_multi_fluid<P>, STEP_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_multi_boundary<P>, STEP_THREADS, 0);
    gf = sms * std::max(1, nf);
    gb = sms * std::max(1, std::min(nb, 2));
}

// Capture the tick: table copies, then per step the fluid and boundary
// launches of both precision groups.
lbm_status capture_tick(lbm_server *s) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    for (int q = 0; q < NGROUPS; ++q)
        cudaMemcpyAsync(s->d_tab[q], s->h_tab[q], sizeof(GroupTable), cudaMemcpyHostToDevice, s->stream);
    cudaMemsetAsync(s->d_flags, 0, NGROUPS * MAX_SLOTS * sizeof(uint32_t), s->stream);
    for (int k = 0; k < s->desc.steps_per_tick; ++k) {
        k_multi_fluid<1><<<s->grid_fluid[0], STEP_THREADS, 0, s->stream>>>(s->d_tab[0], k);
        k_multi_fluid<2><<<s->grid_fluid[1], STEP_THREADS, 0, s->stream>>>(s->d_tab[1], k);
        k_multi_boundary<1><<<s->grid_bnd[0], STEP_THREADS, 0, s->stream>>>(s->d_tab[0], k);
        k_multi_boundary<2><<<s->grid_bnd[1], STEP_THREADS, 0, s->stream>>>(s->d_tab[1], k);
    }
    cudaMemcpyAsync(s->h_flags, s->d_flags, NGROUPS * MAX_SLOTS * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                    s->stream);
    e = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    s->graph_captures += 1;
    return LBM_OK;
}

// The copied flags and the host index are needed only until admission.
void drop_inputs(Request *r) {
    std::vector<uint8_t>().swap(r->flags);
    r->req.flags = nullptr;
    r->idx = HostIndex();
}

void release(lbm_server *s, Request *r) {
    if (r->ctx) {
        lbm_destroy(r->ctx);
        r->ctx = nullptr;
        s->in_use -= r->footprint;
    }
}

lbm_status admit(lbm_server *s, Request *r) {
    lbm_desc d{};
    d.nx = r->req.nx;
    d.ny = r->req.ny;
    d.nz = r->req.nz;
    d.periodic = r->req.periodic;
    d.precision = r->req.precision;
    d.fp16_scale = r->req.fp16_scale;
    d.device = s->desc.device;
    d.stream = s->stream;
    d.allocator = s->desc.allocator;
    lbm_ctx *c = nullptr;
    lbm_status st = lbm_create(&d, &c);
    if (st == LBM_OK) st = ctx_install_index(c, std::move(r->idx));
    if (st == LBM_OK) st = lbm_set_params(c, &r->req.params);
    const double u0[3] = {0.0, 0.0, 0.0};
    if (st == LBM_OK) st = lbm_init_equilibrium(c, 1.0, u0);
    if (st != LBM_OK) {
        r->index_error = c ? lbm_last_error(c) : "context creation failed";
        if (c) lbm_destroy(c);
        drop_inputs(r);
        r->state = LBM_REQ_FAILED;
        r->fail_status = st;
        return st;
    }
    r->ctx = c;
    drop_inputs(r);
    r->group = r->req.precision == LBM_FP16S ? 1 : 0;
    r->state = LBM_REQ_RUNNING;
    s->in_use += r->footprint;
    s->peak = std::max(s->peak, s->in_use);
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_server_create(const lbm_server_desc *desc, lbm_server **out) {
    if (!desc || !out) return LBM_ERR_ARG;
    *out = nullptr;
    if (desc->budget_bytes <= 0 || desc->max_slots < 1 || desc->max_slots > MAX_SLOTS) return LBM_ERR_ARG;
    if (desc->steps_per_tick < 2 || desc->steps_per_tick > 1024 || (desc->steps_per_tick & 1)) return LBM_ERR_ARG;
    if ((desc->allocator.alloc == nullptr) != (desc->allocator.free == nullptr)) return LBM_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    if (desc->device < 0 || desc->device >= ndev) return LBM_ERR_ARG;
    std::unique_ptr<lbm_server> s(new lbm_server());
    s->desc = *desc;
    cudaSetDevice(desc->device);
    // on a failure below, free what was made so far (no worker runs yet)
    auto undo = [&](lbm_status st) {
        for (int q = 0; q < NGROUPS; ++q) {
            if (s->h_tab[q]) cudaFreeHost(s->h_tab[q]);
            if (s->d_tab[q]) cudaFree(s->d_tab[q]);
        }
        if (s->h_flags) cudaFreeHost(s->h_flags);
        if (s->d_flags) cudaFree(s->d_flags);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        cudaGetLastError();
        return st;
    };
    s->stream = static_cast<cudaStream_t>(desc->stream);
    if (!s->stream) {  // graphs cannot be captured on the legacy default stream
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return undo(LBM_ERR_CUDA);
        s->own_stream = true;
    }
    for (int q = 0; q < NGROUPS; ++q) {
        if (cudaMallocHost(&s->h_tab[q], sizeof(GroupTable)) != cudaSuccess) {
            s->h_tab[q] = nullptr;
            return undo(LBM_ERR_CUDA);
        }
        memset(s->h_tab[q], 0, sizeof(GroupTable));
        // the tables are part of the server, not of any lattice: not from the allocator
        if (cudaMalloc(&s->d_tab[q], sizeof(GroupTable)) != cudaSuccess) {
            s->d_tab[q] = nullptr;
            return undo(LBM_ERR_OOM);
        }
    }
    if (cudaMallocHost(&s->h_flags, NGROUPS * MAX_SLOTS * sizeof(uint32_t)) != cudaSuccess) {
        s->h_flags = nullptr;
        return undo(LBM_ERR_CUDA);
    }
    memset(s->h_flags, 0, NGROUPS * MAX_SLOTS * sizeof(uint32_t));
    if (cudaMalloc(&s->d_flags, NGROUPS * MAX_SLOTS * sizeof(uint32_t)) != cudaSuccess) {
        s->d_flags = nullptr;
        return undo(LBM_ERR_OOM);
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, desc->device);
    occupancy_grids<1>(sms, s->grid_fluid[0], s->grid_bnd[0]);
    occupancy_grids<2>(sms, s->grid_fluid[1], s->grid_bnd[1]);
    lbm_server *raw = s.get();
    // Index building is host work that is independent per request: a few
    // threads keep admission fed when many small requests arrive at once.
    const unsigned hw = std::thread::hardware_concurrency();
    const int nworkers = (int)std::max(1u, std::min(4u, hw > 1 ? hw - 1 : 1u));
    for (int k = 0; k < nworkers; ++k) s->workers.emplace_back(worker_loop, raw);
    *out = s.release();
    return LBM_OK;
}

lbm_status lbm_server_destroy(lbm_server *s) {
    if (!s) return LBM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto &w : s->workers)
        if (w.joinable()) w.join();
    cudaSetDevice(s->desc.device);
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->reqs) release(s, kv.second.get());
    if (s->exec) cudaGraphExecDestroy(s->exec);
    for (int q = 0; q < NGROUPS; ++q) {
        if (s->h_tab[q]) cudaFreeHost(s->h_tab[q]);
        if (s->d_tab[q]) cudaFree(s->d_tab[q]);
    }
    if (s->h_flags) cudaFreeHost(s->h_flags);
    if (s->d_flags) cudaFree(s->d_flags);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return LBM_OK;
}

const char *lbm_server_last_error(const lbm_server *s) { return s ? s->err.c_str() : "null server"; }

lbm_status lbm_server_submit(lbm_server *s, const lbm_request *q, int64_t *id) {
    if (!s) return LBM_ERR_ARG;
    if (!id) return sfail(s, LBM_ERR_ARG, "NULL id");
    int64_t active = 0;
    const char *why = "";
    const lbm_status st = check_request(q, s->desc.budget_bytes, &active, &why);
    if (st != LBM_OK) return sfail(s, st, why);
    const int64_t ncell = (int64_t)q->nx * q->ny * q->nz;
    std::unique_ptr<Request> r(new Request());
    r->id = s->next_id++;
    r->req = *q;
    r->flags.assign(q->flags, q->flags + ncell);
    r->req.flags = r->flags.data();
    Request *raw = r.get();
    s->reqs[r->id] = std::move(r);
    s->queue.push_back(raw->id);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->build_queue.push_back(raw);
    }
    s->cv.notify_one();
    *id = raw->id;
    return LBM_OK;
}

lbm_status lbm_server_tick(lbm_server *s, int32_t *running, int32_t *queued) {
    const TraceRange trace("lbm_server_tick");
    if (!s) return LBM_ERR_ARG;
    cudaSetDevice(s->desc.device);
    // retire cancelled lattices
    for (size_t k = 0; k < s->resident.size();) {
        Request *r = s->reqs[s->resident[k]].get();
        if (r->cancel) {
            release(s, r);
            r->state = LBM_REQ_CANCELLED;
            s->resident.erase(s->resident.begin() + k);
        } else {
            ++k;
        }
    }
    // admit requests in submission order (the worker threads may finish the
    // indexes out of order); a request that does not fit the memory left is
    // passed over for later ones that do (first fit)
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request *r = s->reqs[*it].get();
        bool ready;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            ready = r->index_ready;
        }
        if (r->cancel) {
            if (ready) {  // the worker is done with it
                r->state = LBM_REQ_CANCELLED;
                drop_inputs(r);
                it = s->queue.erase(it);
            } else {
                ++it;
            }
            continue;
        }
        if (!ready) break;  // admission keeps submission order: wait for this index
        if (!r->index_error.empty() || r->footprint > s->desc.budget_bytes) {
            r->state = LBM_REQ_FAILED;
            r->fail_status = r->index_error.empty() ? LBM_ERR_OOM : LBM_ERR_ARG;
            drop_inputs(r);
            if (r->index_error.empty()) r->index_error = "footprint exceeds the memory budget";
            it = s->queue.erase(it);
            continue;
        }
        if ((int)s->resident.size() >= s->desc.max_slots) break;
        if (s->in_use + r->footprint > s->desc.budget_bytes) {
            ++it;
            continue;
        }
        if (admit(s, r) == LBM_OK) s->resident.push_back(r->id);
        it = s->queue.erase(it);
    }
    if (running) *running = (int32_t)s->resident.size();
    if (queued) *queued = (int32_t)s->queue.size();
    if (s->resident.empty()) return LBM_OK;

    // per-tick tables
    for (int q = 0; q < NGROUPS; ++q) {
        s->h_tab[q]->n_domains = 0;
        s->h_tab[q]->n_tiles = 0;
        s->h_tab[q]->n_btiles = 0;
    }
    const int K = s->desc.steps_per_tick;
    std::vector<int> steps_now(s->resident.size()), flag_of(s->resident.size());
    for (size_t k = 0; k < s->resident.size(); ++k) {
        Request *r = s->reqs[s->resident[k]].get();
        GroupTable *tab = s->h_tab[r->group];
        flag_of[k] = r->group * MAX_SLOTS + tab->n_domains;
        DomainEntry &e = tab->d[tab->n_domains++];
        ctx_chunk_step_args(r->ctx, &e.a);
        e.a.status = s->d_flags + flag_of[k];  // the lattice's health flag
        e.t_base = r->steps_done;
        e.steps = (int32_t)std::min<int64_t>(K, r->req.steps - r->steps_done);
        steps_now[k] = e.steps;
        e.tile_begin = tab->n_tiles;
        e.btile_begin = tab->n_btiles;
        tab->n_tiles += (int32_t)(((int64_t)e.a.nchunks * CHUNK + STEP_THREADS - 1) / STEP_THREADS);
        tab->n_btiles += (e.a.nbnodes + STEP_THREADS - 1) / STEP_THREADS;
    }
    if (!s->exec) {
        lbm_status st = capture_tick(s);
        if (st != LBM_OK) return st;
    }
    cudaError_t e;
    {
        const TraceRange run("lbm_server_tick: graph");
        e = cudaGraphLaunch(s->exec, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, std::string("tick: ") + cudaGetErrorString(e));
    s->graph_launches += 1;
    s->ticks += 1;
    // account, retire finished lattices
    std::vector<int64_t> still;
    for (size_t k = 0; k < s->resident.size(); ++k) {
        Request *r = s->reqs[s->resident[k]].get();
        ctx_advance(r->ctx, steps_now[k]);
        r->steps_done += steps_now[k];
        s->cell_updates += (double)r->n_active * steps_now[k];
        if (s->h_flags[flag_of[k]]) {  // the tick's health check saw a non-finite cell: evict
            r->state = LBM_REQ_FAILED;
            r->fail_status = LBM_ERR_UNSTABLE;
            r->index_error = "non-finite density or velocity found by the health check at step " +
                             std::to_string(r->steps_done);
            release(s, r);
        } else if (r->steps_done >= r->req.steps) {
            r->rho.assign((size_t)r->n_active, 0.0);
            r->u.assign((size_t)r->n_active * 3, 0.0);
            lbm_status st = lbm_get_moments(r->ctx, r->rho.data(), r->u.data(), LBM_LAYOUT_ACTIVE);
            r->state = st == LBM_OK ? LBM_REQ_DONE : LBM_REQ_FAILED;
            r->fail_status = st;
            if (st != LBM_OK) r->index_error = lbm_last_error(r->ctx);
            release(s, r);
            s->finished += 1;
        } else {
            still.push_back(r->id);
        }
    }
    s->resident.swap(still);
    if (running) *running = (int32_t)s->resident.size();
    return LBM_OK;
}

lbm_status lbm_server_poll(lbm_server *s, int64_t id, int32_t *state, int64_t *steps_done) {
    if (!s) return LBM_ERR_ARG;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_ERR_ARG, "unknown request id");
    if (state) *state = it->second->state;
    if (steps_done) *steps_done = it->second->steps_done;
    return LBM_OK;
}

lbm_status lbm_server_cells(lbm_server *s, int64_t id, int64_t *active_cells) {
    if (!s || !active_cells) return LBM_ERR_ARG;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_ERR_ARG, "unknown request id");
    std::lock_guard<std::mutex> lk(s->mu);
    if (it->second->n_active < 0) return sfail(s, LBM_ERR_STATE, "index not built yet");
    *active_cells = it->second->n_active;
    return LBM_OK;
}

lbm_status lbm_server_result(lbm_server *s, int64_t id, double *rho, double *u) {
    if (!s) return LBM_ERR_ARG;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_ERR_ARG, "unknown request id");
    Request *r = it->second.get();
    if (r->state == LBM_REQ_QUEUED || r->state == LBM_REQ_RUNNING)
        return sfail(s, LBM_ERR_STATE, "request not finished");
    // a terminal request is released here, whatever its outcome (the worker
    // threads are done with it: a request only leaves QUEUED once its index
    // is built)
    if (r->state == LBM_REQ_CANCELLED) {
        s->reqs.erase(it);
        return sfail(s, LBM_ERR_STATE, "request was cancelled");
    }
    if (r->state == LBM_REQ_FAILED) {
        const lbm_status st = r->fail_status != LBM_OK ? r->fail_status : LBM_ERR_ARG;
        const std::string msg = "request failed: " + r->index_error;
        s->reqs.erase(it);
        return sfail(s, st, msg);
    }
    if (rho) memcpy(rho, r->rho.data(), r->rho.size() * 8);
    if (u) memcpy(u, r->u.data(), r->u.size() * 8);
    s->reqs.erase(it);
    return LBM_OK;
}

lbm_status lbm_server_cancel(lbm_server *s, int64_t id) {
    if (!s) return LBM_ERR_ARG;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_ERR_ARG, "unknown request id");
    it->second->cancel = true;
    return LBM_OK;
}

lbm_status lbm_server_info(lbm_server *s, double out[8]) {
    if (!s || !out) return LBM_ERR_ARG;
    out[0] = s->cell_updates;
    out[1] = s->ticks;
    out[2] = (double)s->in_use;
    out[3] = (double)s->peak;
    out[4] = s->graph_launches;
    out[5] = s->graph_captures;
    out[6] = s->finished;
    out[7] = (double)s->queue.size();
    return LBM_OK;
}

lbm_status lbm_server_check_request(const lbm_request *req, int64_t budget_bytes, int64_t out[4],
                                    const char **why) {
    static thread_local std::string msg;
    const char *w = "";
    int64_t active = 0;
    if (out) out[0] = out[1] = out[2] = out[3] = 0;
    lbm_status st = check_request(req, budget_bytes, &active, &w);
    if (st == LBM_OK) {
        HostIndex idx;
        msg = build_index(req->flags, req->nx, req->ny, req->nz, req->periodic, idx, MAX_SLOTS_32);
        if (!msg.empty()) {
            st = LBM_ERR_ARG;
            w = msg.c_str();
        } else {
            const int64_t fp = request_footprint(*req, idx);
            if (out) {
                out[0] = idx.n_active;
                out[1] = idx.nslots;
                out[2] = fp;
                out[3] = (int64_t)idx.bnodes.size();
            }
            if (fp > budget_bytes) {
                st = LBM_ERR_OOM;
                w = "footprint exceeds the memory budget";
            }
        }
    }
    if (why) *why = w;
    return st;
}

}  // extern "C"
