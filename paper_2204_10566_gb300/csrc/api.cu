// C ABI of the lattice Boltzmann library (declared in include/lbm.h): context
// management, device memory, parameter derivation, and the step loop.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
// Per-cell (rho, u) in active order -> rho[n], u[n][3] on the device (common.cu).
cudaError_t launch_split_moments(const double *in, int64_t n, double *rho, double *u, cudaStream_t s);
}  // namespace lbm

using namespace lbm;

struct lbm_ctx {
    lbm_desc desc{};
    cudaStream_t stream = nullptr;
    std::string err;
    bool has_geom = false, has_params = false, has_state = false;
    HostIndex idx;
    // device buffers
    void *f[2] = {nullptr, nullptr};      // population buffers (inside the raw allocations)
    void *f_raw[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t *d_mask = nullptr;           // link words (inside d_mask_raw)
    uint32_t *d_mask_raw = nullptr;
    int4 *d_row_nb = nullptr;
    int2 *d_chunks = nullptr;
    int4 *d_bnodes = nullptr;
    int32_t *d_slot_of_active = nullptr;
    int32_t *d_wall_qidx = nullptr;  // per slot: wall-distance record or -1 (lbm_set_wall_q)
    uint8_t *d_wall_q = nullptr;     // 32-byte records
    int64_t n_wall_q = 0;
    int4 *d_wnodes = nullptr;        // cells with interpolated walls, out of the chunk lanes
    int64_t n_wnodes = 0;
    int2 *d_chunks_wall = nullptr;   // chunk records without those cells (the fluid kernel's list)
    int32_t *d_tiles_wall = nullptr; // tile records without those cells
    int64_t n_tiles_wall = 0;
    int2 *d_items_wall = nullptr;    // their pair-kernel items
    int64_t n_items_wall = 0;
    int2 *d_rest_wall = nullptr;     // and the chunks beside those items
    int64_t n_rest_wall = 0;
    bool wide_offsets = false;       // LBM_WIDE_OFFSETS=1 at creation: the 64-bit offset kernels always
    FluidKernel fluid_kernel = FluidKernel::AUTO;  // LBM_FLUID_KERNEL at creation
    SideStream side;                 // the wall-cell and inlet/outlet kernels beside the fluid kernel
    int32_t *d_tiles = nullptr;      // tile records of the tile fluid kernel
    int2 *d_items = nullptr;         // pairs of fast tiles of the FP16S pair kernel
    int2 *d_rest = nullptr;          // chunks of the other tiles (the chunk kernel beside it)
    double *d_partials = nullptr;
    double *d_health = nullptr;
    uint32_t *d_status = nullptr;
    double *d_stats = nullptr;
    int nblocks = 0;        // partial-sum capacity (blocks)
    int fluid_blocks = 0;   // blocks of the chunk fluid kernel
    int64_t device_bytes = 0;
    int64_t kernel_launches = 0;  // kernels lbm_step has launched on this context
    // parameters and state
    lbm_params params{};
    double omega = 0.0;
    bool ghost1 = true;
    int prefetch_ahead = 0, prefetch_key = -1;  // L2 prefetch lookahead of the fluid kernel, per variant
    int64_t t = 0;
    int64_t check_every = 0;
    bool stats_on = false;
    int64_t stats_stride = 1, stats_start = 0, stats_samples = 0;
    int32_t stats_mode = LBM_STATS_AXIAL;  // what lbm_stats_begin allocates
    int stats_ncomp = 0;                   // accumulator rows of d_stats (0: none)
    double health[6] = {0, 0, 0, 0, 0, 0};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what) {
    return fail(c, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

int storage_bytes(int precision) { return precision == LBM_FP64 ? 8 : (precision == LBM_FP32 ? 4 : 2); }

void *dev_alloc(lbm_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (c->desc.allocator.alloc) {
        p = c->desc.allocator.alloc(bytes, c->desc.allocator.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->device_bytes += (int64_t)bytes;
    return p;
}

void dev_free(lbm_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    c->device_bytes -= (int64_t)bytes;
    if (c->desc.allocator.alloc)
        c->desc.allocator.free(p, c->desc.allocator.user);
    else
        cudaFree(p);
}

size_t pop_bytes(const lbm_ctx *c) { return (size_t)27 * (size_t)c->idx.nslots * storage_bytes(c->desc.precision); }
size_t margin_bytes(const lbm_ctx *c) { return (size_t)buffer_margin(c->idx.n_row) * storage_bytes(c->desc.precision); }
size_t raw_pop_bytes(const lbm_ctx *c) { return pop_bytes(c) + 2 * margin_bytes(c); }
size_t raw_mask_bytes(const lbm_ctx *c) { return ((size_t)c->idx.nslots + 2 * MASK_MARGIN) * 4; }

void release_wall_q(lbm_ctx *c) {
    dev_free(c, c->d_wall_qidx, (size_t)c->idx.nslots * 4);
    dev_free(c, c->d_wall_q, (size_t)c->n_wall_q * 32);
    dev_free(c, c->d_wnodes, (size_t)c->n_wnodes * 16);
    if (c->d_chunks_wall) dev_free(c, c->d_chunks_wall, c->idx.chunks.size() * 8);
    if (c->d_tiles_wall) dev_free(c, c->d_tiles_wall, (size_t)c->n_tiles_wall * TILE_INTS * 4);
    if (c->d_items_wall) dev_free(c, c->d_items_wall, (size_t)c->n_items_wall * 8);
    if (c->d_rest_wall) dev_free(c, c->d_rest_wall, (size_t)c->n_rest_wall * 8);
    c->d_items_wall = nullptr;
    c->n_items_wall = 0;
    c->d_rest_wall = nullptr;
    c->n_rest_wall = 0;
    c->d_chunks_wall = nullptr;
    c->d_tiles_wall = nullptr;
    c->n_tiles_wall = 0;
    c->d_wall_qidx = nullptr;
    c->d_wall_q = nullptr;
    c->d_wnodes = nullptr;
    c->n_wall_q = 0;
    c->n_wnodes = 0;
}

void release_geometry(lbm_ctx *c) {
    const size_t ns = (size_t)c->idx.nslots;
    dev_free(c, c->f_raw[0], raw_pop_bytes(c));
    dev_free(c, c->f_raw[1], raw_pop_bytes(c));
    dev_free(c, c->d_mask_raw, raw_mask_bytes(c));
    dev_free(c, c->d_row_nb, c->idx.row_nb.size() * 4);
    dev_free(c, c->d_chunks, c->idx.chunks.size() * 8);
    dev_free(c, c->d_bnodes, c->idx.bnodes.size() * 16);
    dev_free(c, c->d_slot_of_active, c->idx.slot_of_active.size() * 4);
    dev_free(c, c->d_tiles, c->idx.tiles.size() * 4);
    dev_free(c, c->d_items, c->idx.pair_items.size() * 8);
    dev_free(c, c->d_rest, c->idx.rest_chunks.size() * 8);
    c->d_tiles = nullptr;
    c->d_items = nullptr;
    c->d_rest = nullptr;
    release_wall_q(c);
    dev_free(c, c->d_partials, (size_t)c->nblocks * REDUCE_SLOTS * 8);
    dev_free(c, c->d_health, 8 * 8);
    dev_free(c, c->d_status, 256);
    dev_free(c, c->d_stats, (size_t)c->stats_ncomp * ns * 8);
    c->f[0] = c->f[1] = nullptr;
    c->f_raw[0] = c->f_raw[1] = nullptr;
    c->d_mask = c->d_mask_raw = nullptr;
    c->d_row_nb = nullptr;
    c->d_chunks = nullptr;
    c->d_bnodes = nullptr;
    c->d_slot_of_active = nullptr;
    c->d_partials = nullptr;
    c->d_health = nullptr;
    c->d_status = nullptr;
    c->d_stats = nullptr;
    c->stats_ncomp = 0;
    c->has_geom = c->has_state = false;
}

size_t stats_bytes(const lbm_ctx *c) { return (size_t)c->stats_ncomp * (size_t)c->idx.nslots * 8; }

float fp16_scale(const lbm_ctx *c) { return c->desc.precision == LBM_FP16S ? c->desc.fp16_scale : 1.0f; }

// Dispatch a launcher over the storage precision.
#define DISPATCH(prec, fn, ...)                                   \
    ((prec) == LBM_FP64 ? fn<0>(__VA_ARGS__)                      \
                        : ((prec) == LBM_FP32 ? fn<1>(__VA_ARGS__) : fn<2>(__VA_ARGS__)))

// Host arrays <-> active order.
int64_t layout_count(const lbm_ctx *c, int32_t layout) {
    return layout == LBM_LAYOUT_BOX ? (int64_t)c->desc.nx * c->desc.ny * c->desc.nz : c->idx.n_active;
}

template <class F>
void for_active(const lbm_ctx *c, int32_t layout, F fn) {  // fn(active k, host row)
    for (int64_t k = 0; k < c->idx.n_active; ++k) fn(k, layout == LBM_LAYOUT_BOX ? c->idx.box_of_active[k] : k);
}

lbm_status need(lbm_ctx *c, bool geom, bool params, bool state) {
    if (!c) return LBM_ERR_ARG;
    if (geom && !c->has_geom) return fail(c, LBM_ERR_STATE, "no geometry: call lbm_set_geometry first");
    if (params && !c->has_params) return fail(c, LBM_ERR_STATE, "no parameters: call lbm_set_params first");
    if (state && !c->has_state) return fail(c, LBM_ERR_STATE, "no state: call an init function first");
    c->err.clear();
    return LBM_OK;
}

// Whether the row axis of the context's index is periodic.
int periodic_rows(const lbm_ctx *c) {
    return (c->desc.periodic & (c->idx.row_axis == 2 ? LBM_PERIODIC_Z : LBM_PERIODIC_X)) ? 1 : 0;
}

// Whether the next steps run the tile fluid kernel (default ghost rates,
// 32-bit offsets; FP32 by default, FP16S when LBM_FLUID_KERNEL asks for the
// tile or the pair kernel), and the partial sums the step kernels write: the
// fluid kernel's blocks, then the inlet/outlet blocks, then the wall-cell
// blocks.
bool wide_offsets(const lbm_ctx *c) { return c->wide_offsets || c->idx.nslots > MAX_SLOTS_32; }
int64_t tile_count(const lbm_ctx *c) {
    return c->d_tiles_wall ? c->n_tiles_wall : (int64_t)c->idx.tiles.size() / TILE_INTS;
}
bool tiled(const lbm_ctx *c) {
    const FluidKernel k = c->fluid_kernel;
    const bool wanted = k == FluidKernel::TILE || k == FluidKernel::PAIRS ||
                        (k == FluidKernel::AUTO && c->desc.precision == LBM_FP32);
    return wanted && c->desc.precision != LBM_FP64 && c->ghost1 && !wide_offsets(c) && tile_count(c) > 0;
}
// LBM_FLUID_KERNEL=pairs splits the FP16S fluid cells: pairs of fast tiles
// run on the pair kernel, the chunks of every other tile on the chunk kernel.
bool pairs(const lbm_ctx *c) { return c->desc.precision == LBM_FP16S && c->fluid_kernel == FluidKernel::PAIRS; }
int64_t item_count(const lbm_ctx *c) {
    return c->d_tiles_wall ? c->n_items_wall : (int64_t)c->idx.pair_items.size();
}
int64_t rest_count(const lbm_ctx *c) {
    return c->d_tiles_wall ? c->n_rest_wall : (int64_t)c->idx.rest_chunks.size();
}
int split_blocks(int64_t rest, int64_t items) { return fluid_blocks((int32_t)rest) + tile_blocks(items); }
int fluid_partials(const lbm_ctx *c) {
    if (!tiled(c)) return c->fluid_blocks;
    return pairs(c) ? split_blocks(rest_count(c), item_count(c)) : tile_blocks(tile_count(c));
}
int step_partials(const lbm_ctx *c) {
    return fluid_partials(c) + node_blocks((int64_t)c->idx.bnodes.size()) + node_blocks(c->n_wnodes);
}
// Partial-sum capacity for either fluid kernel, the wall cells and lbm_get_totals.
int partial_capacity(const lbm_ctx *c, int64_t n_wnodes) {
    const int nodes = node_blocks((int64_t)c->idx.bnodes.size()) + node_blocks(n_wnodes);
    const int tiles = tile_blocks(std::max<int64_t>((int64_t)c->idx.tiles.size() / TILE_INTS, c->n_tiles_wall));
    const int split = std::max(split_blocks((int64_t)c->idx.rest_chunks.size(), (int64_t)c->idx.pair_items.size()),
                               split_blocks(c->n_rest_wall, c->n_items_wall));
    return std::max({c->fluid_blocks + nodes, tiles + nodes, split + nodes, node_blocks(c->idx.n_active)});
}

// Ghost slots and periodic copies of the current buffer from its active cells.
cudaError_t fill_ghosts(lbm_ctx *c) {
    return DISPATCH(c->desc.precision, launch_fill_ghosts, c->f[c->cur], c->d_mask, c->d_chunks, c->d_row_nb,
                    (int32_t)c->idx.chunks.size(), c->d_bnodes, (int32_t)c->idx.bnodes.size(), c->idx.nslots,
                    c->idx.n_row, periodic_rows(c), c->idx.row_axis, c->stream);
}

lbm_status reset_state(lbm_ctx *c) {
    CK(fill_ghosts(c), "fill ghost slots");
    c->t = 0;
    c->stats_samples = 0;
    c->stats_on = false;
    CK(cudaMemsetAsync(c->d_status, 0, 4, c->stream), "reset status");
    if (c->d_stats) CK(cudaMemsetAsync(c->d_stats, 0, stats_bytes(c), c->stream), "reset stats");
    c->has_state = true;
    return LBM_OK;
}

}  // namespace

namespace lbm {

// Everything a step kernel needs from a context; fin/fout/t_new describe
// the next step from the current state, flags are cleared.
void ctx_step_args(lbm_ctx *c, StepArgs *out) {
    StepArgs a{};
    a.mask = c->d_mask;
    a.row_nb = c->d_row_nb;
    a.chunks = c->d_chunks_wall ? c->d_chunks_wall : c->d_chunks;
    a.stride = c->idx.nslots;
    a.nchunks = (int32_t)c->idx.chunks.size();
    a.bnodes = c->d_bnodes;
    a.nbnodes = (int32_t)c->idx.bnodes.size();
    a.fluid_blocks = fluid_partials(c);
    a.status = c->d_status;
    a.nx = c->desc.nx;
    a.ny = c->desc.ny;
    a.nz = c->desc.nz;
    a.na_e = c->idx.na_e;
    a.n_row = c->idx.n_row;
    a.row_axis = c->idx.row_axis;
    a.periodic_row = periodic_rows(c);
    a.profile = c->params.inlet_profile;
    a.inlet_ramp = c->params.inlet_ramp;
    const double gr[4] = {c->params.omega3, c->params.omega4, c->params.omega5, c->params.omega6};
    a.pd.omega = c->omega;
    for (int q = 0; q < 4; ++q) a.pd.ghost[q] = gr[q];
    a.pd.u_in = c->params.u_in;
    a.pd.d_in = c->params.d_in;
    a.pd.axis_x = c->params.axis_x;
    a.pd.axis_y = c->params.axis_y;
    a.pd.noise_amp = c->params.noise_amp;
    a.pd.rho_out = c->params.rho_out;
    a.pf.omega = (float)a.pd.omega;
    for (int q = 0; q < 4; ++q) a.pf.ghost[q] = (float)gr[q];
    a.pf.u_in = (float)a.pd.u_in;
    a.pf.d_in = (float)a.pd.d_in;
    a.pf.axis_x = (float)a.pd.axis_x;
    a.pf.axis_y = (float)a.pd.axis_y;
    a.pf.noise_amp = (float)a.pd.noise_amp;
    a.pf.rho_out = (float)a.pd.rho_out;
    a.seed = c->params.noise_seed;
    a.scale = fp16_scale(c);
    a.inv_scale = 1.0f / a.scale;
    a.stats = c->d_stats;
    a.partials = c->d_partials;
    a.wide_offsets = c->wide_offsets ? 1 : 0;
    const bool wide = wide_offsets(c);
    if (tiled(c)) {
        a.tiles = c->d_tiles_wall ? c->d_tiles_wall : c->d_tiles;
        a.ntiles = (int32_t)tile_count(c);
        if (pairs(c)) {  // the chunk kernel takes the rest chunks
            a.items = c->d_tiles_wall ? c->d_items_wall : c->d_items;
            a.nitems = (int32_t)item_count(c);
            a.chunks = c->d_tiles_wall ? c->d_rest_wall : c->d_rest;
            a.nchunks = (int32_t)rest_count(c);
        }
    }
    const int key = (c->ghost1 ? 2 : 0) + (wide ? 1 : 0);
    if (c->prefetch_key != key) {
        c->prefetch_ahead = DISPATCH(c->desc.precision, step_prefetch_ahead, c->ghost1, wide, c->desc.device);
        c->prefetch_key = key;
    }
    a.prefetch_ahead = c->prefetch_ahead;
    a.wall_qidx = c->d_wall_qidx;
    a.wall_q = c->d_wall_q;
    a.wnodes = c->d_wnodes;
    a.nwnodes = (int32_t)c->n_wnodes;
    a.fin = c->f[c->cur];
    a.fout = c->f[1 - c->cur];
    a.t_new = c->t + 1;
    a.flags = 0;
    *out = a;
}

// The same arguments for the chunk kernel's view of the lattice (every chunk,
// every inlet/outlet node, no tiles, no pair items): the request server's
// multi-lattice kernels walk the lattice that way whatever fluid kernel the
// context's own steps run.
void ctx_chunk_step_args(lbm_ctx *c, StepArgs *out) {
    ctx_step_args(c, out);
    out->chunks = c->d_chunks_wall ? c->d_chunks_wall : c->d_chunks;
    out->nchunks = (int32_t)c->idx.chunks.size();
    out->bnodes = c->d_bnodes;
    out->nbnodes = (int32_t)c->idx.bnodes.size();
    out->tiles = nullptr;
    out->ntiles = 0;
    out->items = nullptr;
    out->nitems = 0;
    out->fluid_blocks = c->fluid_blocks;
}

void ctx_advance(lbm_ctx *c, int64_t steps) {
    c->t += steps;
    if (steps & 1) c->cur = 1 - c->cur;
}

int64_t ctx_steps(const lbm_ctx *c) { return c->t; }
int64_t ctx_device_bytes(const lbm_ctx *c) { return c->device_bytes; }
bool ctx_ready(const lbm_ctx *c) { return c->has_geom && c->has_params && c->has_state; }
bool ctx_ghost1(const lbm_ctx *c) { return c->ghost1; }
int ctx_precision(const lbm_ctx *c) { return c->desc.precision; }
int64_t ctx_slots(const lbm_ctx *c) { return c->idx.nslots; }

// FP16S scale of a descriptor: 0 selects the default 4096, any other value
// must be a positive power of two (so that scaling is exact).  Returns the
// scale, or 0 when the value is invalid.
float resolve_fp16_scale(float s) {
    if (s == 0.0f) return 4096.0f;
    int ex;
    return (s > 0.0f && std::frexp(s, &ex) == 0.5f) ? s : 0.0f;
}

}  // namespace lbm

extern "C" {

const char *lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_ARG: return "invalid argument";
        case LBM_ERR_OOM: return "out of device memory";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_STATE: return "call out of order";
        case LBM_ERR_UNSTABLE: return "non-finite state";
        case LBM_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

void lbm_params_default(lbm_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->omega3 = p->omega4 = p->omega5 = p->omega6 = 1.0;
    p->inlet_profile = LBM_PROFILE_PLUG;
    p->axis_x = p->axis_y = -1.0;
    p->rho_out = 1.0;
}

lbm_status lbm_create(const lbm_desc *desc, lbm_ctx **out) {
    if (!desc || !out) return LBM_ERR_ARG;
    *out = nullptr;
    if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1) return LBM_ERR_ARG;
    if ((int64_t)desc->nx * desc->ny * desc->nz > ((int64_t)1 << 40)) return LBM_ERR_ARG;
    if (desc->precision < LBM_FP64 || desc->precision > LBM_FP16S) return LBM_ERR_ARG;
    if (desc->periodic & ~7) return LBM_ERR_ARG;
    if ((desc->allocator.alloc == nullptr) != (desc->allocator.free == nullptr)) return LBM_ERR_ARG;
    if (desc->row_axis != LBM_ROWS_AUTO && desc->row_axis != LBM_ROWS_X && desc->row_axis != LBM_ROWS_Z)
        return LBM_ERR_ARG;
    const float s = resolve_fp16_scale(desc->fp16_scale);
    if (s == 0.0f) return LBM_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    if (desc->device < 0 || desc->device >= ndev) return LBM_ERR_ARG;
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OOM;
    c->desc = *desc;
    c->desc.fp16_scale = s;
    c->stream = static_cast<cudaStream_t>(desc->stream);
    // Lattices of 2^32 / 27 slots or more need 64-bit element offsets; this
    // switch runs those kernels on any lattice, so that tests can cover them
    // without allocating tens of gigabytes.
    const char *wide = std::getenv("LBM_WIDE_OFFSETS");
    c->wide_offsets = wide && wide[0] == '1';
    // LBM_FLUID_KERNEL selects another fluid kernel than the default (FP32:
    // tile kernel, FP16S / FP64: chunk kernel), for testing every variant on
    // the same lattices: "chunk", "tile" or "pairs" (FP16S pair + chunk kernel)
    const char *fk = std::getenv("LBM_FLUID_KERNEL");
    if (fk && std::strcmp(fk, "chunk") == 0) c->fluid_kernel = FluidKernel::CHUNK;
    if (fk && std::strcmp(fk, "tile") == 0) c->fluid_kernel = FluidKernel::TILE;
    if (fk && std::strcmp(fk, "pairs") == 0) c->fluid_kernel = FluidKernel::PAIRS;
    lbm_params_default(&c->params);
    {
        // a second stream (at the highest priority) and two events, so that
        // each step can run its wall-cell and inlet/outlet kernels beside the
        // fluid kernel; without them (or with LBM_SIDE_STREAM=0 at creation,
        // for tests) the step runs its kernels in sequence on one stream
        DeviceGuard g(c->desc.device);
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) hi = 0;
        const char *ss = std::getenv("LBM_SIDE_STREAM");
        const bool ok = !(ss && ss[0] == '0') && cudaStreamCreateWithPriority(&c->side.stream, cudaStreamNonBlocking, hi) == cudaSuccess &&
                        cudaEventCreateWithFlags(&c->side.fork, cudaEventDisableTiming) == cudaSuccess &&
                        cudaEventCreateWithFlags(&c->side.join, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            if (c->side.stream) cudaStreamDestroy(c->side.stream);
            if (c->side.fork) cudaEventDestroy(c->side.fork);
            c->side = SideStream{};
        }
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx *c) {
    if (!c) return LBM_OK;
    DeviceGuard g(c->desc.device);
    cudaStreamSynchronize(c->stream);
    release_geometry(c);
    if (c->side.stream) {
        cudaStreamSynchronize(c->side.stream);
        cudaStreamDestroy(c->side.stream);
    }
    if (c->side.fork) cudaEventDestroy(c->side.fork);
    if (c->side.join) cudaEventDestroy(c->side.join);
    delete c;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c) { return c ? c->err.c_str() : "null context"; }

lbm_status lbm_set_wall_q(lbm_ctx *c, const int64_t *cells, const uint8_t *q, int64_t n) {
    const TraceRange trace("lbm_set_wall_q");
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (n < 0 || (n > 0 && (!cells || !q))) return fail(c, LBM_ERR_ARG, "bad wall-distance arrays");
    DeviceGuard g(c->desc.device);
    CK(cudaStreamSynchronize(c->stream), "sync before wall distances");
    release_wall_q(c);
    if (n == 0) return LBM_OK;
    const int64_t ncell = (int64_t)c->desc.nx * c->desc.ny * c->desc.nz;
    // box index -> active index, to find each cell's slot
    std::vector<int64_t> active_of_box((size_t)ncell, -1);
    for (int64_t k = 0; k < c->idx.n_active; ++k) active_of_box[(size_t)c->idx.box_of_active[k]] = k;
    std::vector<int32_t> qidx((size_t)c->idx.nslots, -1);
    std::vector<uint8_t> rec((size_t)n * 32, 128);
    for (int64_t r = 0; r < n; ++r) {
        const int64_t b = cells[r];
        if (b < 0 || b >= ncell || active_of_box[(size_t)b] < 0)
            return fail(c, LBM_ERR_ARG, "wall-distance record " + std::to_string(r) + " is not an active cell");
        const int32_t slot = c->idx.slot_of_active[(size_t)active_of_box[(size_t)b]];
        if (((c->idx.mask[(size_t)slot] >> TYPE_SHIFT) & 3u) != TYPE_FLUID)
            return fail(c, LBM_ERR_ARG, "wall-distance record " + std::to_string(r) + " is not a fluid cell");
        if (qidx[(size_t)slot] >= 0)
            return fail(c, LBM_ERR_ARG, "cell listed twice in the wall distances");
        for (int i = 0; i < 27; ++i)
            if (q[r * 27 + i] == 0) return fail(c, LBM_ERR_ARG, "wall distance q = 0 (a wall through a cell centre)");
        qidx[(size_t)slot] = (int32_t)r;
        memcpy(&rec[(size_t)r * 32], q + r * 27, 27);
    }
    // cells with at least one interpolated link leave the chunk lanes for the
    // wall kernel's list (slot order)
    const bool zrows = c->idx.row_axis == 2;
    std::vector<int4> wn;
    std::vector<int2> chunks = c->idx.chunks;
    std::vector<char> is_wall((size_t)c->idx.nslots, 0);
    for (int64_t r = 0; r < n; ++r) {
        bool interp = false;
        for (int i = 0; i < 27; ++i) interp |= q[r * 27 + i] != 128;
        if (!interp) continue;
        const int64_t b = cells[r];
        const int x = (int)(b % c->desc.nx), y = (int)((b / c->desc.nx) % c->desc.ny);
        const int z = (int)(b / ((int64_t)c->desc.nx * c->desc.ny));
        // storage coordinates: p along the rows, (a, b) across them
        const int p = zrows ? z : x, ra = zrows ? x : y, rb = zrows ? y : z;
        const int row = (ra + 1) + c->idx.na_e * (rb + 1);
        const int32_t slot = c->idx.slot_of_active[(size_t)active_of_box[(size_t)b]];
        wn.push_back(make_int4(p, row, slot, (int)r));
        is_wall[(size_t)slot] = 1;
    }
    std::sort(wn.begin(), wn.end(), [](const int4 &p, const int4 &q2) { return p.z < q2.z; });
    for (int2 &ch : chunks) {
        const int x0 = (int)((uint32_t)ch.y & CHUNK_X0_MASK);
        const int32_t base = c->idx.row_nb[(size_t)ch.x * ROW_RECORD_INTS + 4];
        uint32_t lanes = ((uint32_t)ch.y >> CHUNK_LANES_SHIFT) & 0xFFu;
        for (int l = 0; l < CHUNK; ++l)
            if (((lanes >> l) & 1u) && is_wall[(size_t)(base + x0 + l)]) lanes &= ~(1u << l);
        ch.y = (int)((uint32_t)x0 | (lanes << CHUNK_LANES_SHIFT));
    }
    const std::vector<int32_t> tiles =
        wn.empty() ? std::vector<int32_t>()
                   : build_tiles(chunks, c->idx.row_nb, c->idx.mask, c->idx.n_row, periodic_rows(c) != 0);
    const std::vector<int2> items = build_pair_items(tiles);
    const std::vector<int2> rest = build_rest_chunks(chunks, tiles, items);
    c->d_wall_qidx = (int32_t *)dev_alloc(c, qidx.size() * 4);
    c->d_wall_q = (uint8_t *)dev_alloc(c, rec.size());
    c->n_wall_q = n;
    c->n_wnodes = (int64_t)wn.size();
    c->d_wnodes = wn.empty() ? nullptr : (int4 *)dev_alloc(c, wn.size() * 16);
    if (!wn.empty()) c->d_chunks_wall = (int2 *)dev_alloc(c, chunks.size() * 8);
    if (!wn.empty()) {
        c->n_tiles_wall = (int64_t)tiles.size() / TILE_INTS;
        c->d_tiles_wall = (int32_t *)dev_alloc(c, tiles.size() * 4);
        c->n_items_wall = (int64_t)items.size();
        c->d_items_wall = (int2 *)dev_alloc(c, items.size() * 8);
        c->n_rest_wall = (int64_t)rest.size();
        c->d_rest_wall = (int2 *)dev_alloc(c, rest.size() * 8);
    }
    const int capacity = partial_capacity(c, c->n_wnodes);
    double *partials = c->d_partials;
    if (capacity > c->nblocks) {  // room for the wall kernel's partial sums
        partials = (double *)dev_alloc(c, (size_t)capacity * REDUCE_SLOTS * 8);
        if (partials) {
            dev_free(c, c->d_partials, (size_t)c->nblocks * REDUCE_SLOTS * 8);
            c->d_partials = partials;
            c->nblocks = capacity;
        }
    }
    if (!c->d_wall_qidx || !c->d_wall_q ||
        (!wn.empty() && (!c->d_wnodes || !c->d_chunks_wall || !c->d_tiles_wall || !c->d_items_wall ||
                         !c->d_rest_wall)) ||
        !partials) {
        release_wall_q(c);
        return fail(c, LBM_ERR_OOM, "wall-distance allocation failed");
    }
    CK(cudaMemcpyAsync(c->d_wall_qidx, qidx.data(), qidx.size() * 4, cudaMemcpyHostToDevice, c->stream),
       "copy wall index");
    CK(cudaMemcpyAsync(c->d_wall_q, rec.data(), rec.size(), cudaMemcpyHostToDevice, c->stream), "copy wall records");
    if (!wn.empty())
        CK(cudaMemcpyAsync(c->d_wnodes, wn.data(), wn.size() * 16, cudaMemcpyHostToDevice, c->stream),
           "copy wall cells");
    if (!wn.empty())
        CK(cudaMemcpyAsync(c->d_chunks_wall, chunks.data(), chunks.size() * 8, cudaMemcpyHostToDevice, c->stream),
           "copy chunk lanes");
    if (!tiles.empty())
        CK(cudaMemcpyAsync(c->d_tiles_wall, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice, c->stream),
           "copy tile records");
    if (!items.empty())
        CK(cudaMemcpyAsync(c->d_items_wall, items.data(), items.size() * 8, cudaMemcpyHostToDevice, c->stream),
           "copy pair items");
    if (!rest.empty())
        CK(cudaMemcpyAsync(c->d_rest_wall, rest.data(), rest.size() * 8, cudaMemcpyHostToDevice, c->stream),
           "copy rest chunks");
    CK(cudaStreamSynchronize(c->stream), "sync wall distances");
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx *c, const uint8_t *flags) {
    const TraceRange trace("lbm_set_geometry");
    if (!c) return LBM_ERR_ARG;
    if (!flags) return fail(c, LBM_ERR_ARG, "flags is NULL");
    HostIndex idx;
    std::string msg = build_index(flags, c->desc.nx, c->desc.ny, c->desc.nz, c->desc.periodic, idx, 0,
                                  c->desc.row_axis);
    if (!msg.empty()) return fail(c, LBM_ERR_ARG, msg);
    return lbm::ctx_install_index(c, std::move(idx));
}

}  // extern "C"

namespace lbm {

int64_t ctx_footprint(const lbm_desc &d, const HostIndex &ix) {
    const int S = storage_bytes(d.precision);
    const int64_t pop = 27 * ix.nslots * S + 2 * buffer_margin(ix.n_row) * S;
    const int64_t blocks = std::max<int64_t>(fluid_blocks((int32_t)ix.chunks.size()) + node_blocks((int64_t)ix.bnodes.size()),
                                             node_blocks(ix.n_active));
    return 2 * pop + (ix.nslots + 2 * MASK_MARGIN) * 4 + (int64_t)ix.row_nb.size() * 4 + (int64_t)ix.chunks.size() * 8 +
           (int64_t)ix.bnodes.size() * 16 + ix.n_active * 4 + (int64_t)ix.tiles.size() * 4 +
           (int64_t)ix.pair_items.size() * 8 + (int64_t)ix.rest_chunks.size() * 8 +
           blocks * REDUCE_SLOTS * 8 + 64 + 256;
}

lbm_status ctx_install_index(lbm_ctx *c, HostIndex &&idx) {
    DeviceGuard g(c->desc.device);
    CK(cudaStreamSynchronize(c->stream), "sync before geometry change");
    release_geometry(c);
    c->idx = std::move(idx);
    const size_t ns = (size_t)c->idx.nslots;
    c->fluid_blocks = DISPATCH(c->desc.precision, step_fluid_blocks, (int32_t)c->idx.chunks.size());
    c->nblocks = partial_capacity(c, 0);
    for (int k = 0; k < 2; ++k) {
        c->f_raw[k] = dev_alloc(c, raw_pop_bytes(c));
        c->f[k] = c->f_raw[k] ? static_cast<char *>(c->f_raw[k]) + margin_bytes(c) : nullptr;
    }
    c->d_mask_raw = (uint32_t *)dev_alloc(c, raw_mask_bytes(c));
    c->d_mask = c->d_mask_raw ? c->d_mask_raw + MASK_MARGIN : nullptr;
    c->d_row_nb = (int4 *)dev_alloc(c, c->idx.row_nb.size() * 4);
    c->d_chunks = (int2 *)dev_alloc(c, c->idx.chunks.size() * 8);
    c->d_bnodes = (int4 *)dev_alloc(c, c->idx.bnodes.size() * 16);
    c->d_slot_of_active = (int32_t *)dev_alloc(c, c->idx.slot_of_active.size() * 4);
    c->d_tiles = (int32_t *)dev_alloc(c, c->idx.tiles.size() * 4);
    c->d_items = (int2 *)dev_alloc(c, c->idx.pair_items.size() * 8);
    c->d_rest = (int2 *)dev_alloc(c, c->idx.rest_chunks.size() * 8);
    c->d_partials = (double *)dev_alloc(c, (size_t)c->nblocks * REDUCE_SLOTS * 8);
    c->d_health = (double *)dev_alloc(c, 8 * 8);
    c->d_status = (uint32_t *)dev_alloc(c, 256);
    if (!c->f[0] || !c->f[1] || !c->d_mask || !c->d_row_nb || !c->d_chunks || !c->d_bnodes || !c->d_slot_of_active ||
        !c->d_tiles || !c->d_items || !c->d_rest || !c->d_partials || !c->d_health || !c->d_status) {
        release_geometry(c);
        return fail(c, LBM_ERR_OOM, "device allocation failed in lbm_set_geometry");
    }
    CK(cudaMemsetAsync(c->d_mask_raw, 0, raw_mask_bytes(c), c->stream), "clear link words");
    CK(cudaMemcpyAsync(c->d_mask, c->idx.mask.data(), ns * 4, cudaMemcpyHostToDevice, c->stream), "copy mask");
    CK(cudaMemcpyAsync(c->d_row_nb, c->idx.row_nb.data(), c->idx.row_nb.size() * 4, cudaMemcpyHostToDevice,
                       c->stream),
       "copy row records");
    CK(cudaMemcpyAsync(c->d_chunks, c->idx.chunks.data(), c->idx.chunks.size() * 8, cudaMemcpyHostToDevice,
                       c->stream),
       "copy chunks");
    if (!c->idx.bnodes.empty())
        CK(cudaMemcpyAsync(c->d_bnodes, c->idx.bnodes.data(), c->idx.bnodes.size() * 16, cudaMemcpyHostToDevice,
                           c->stream),
           "copy boundary nodes");
    CK(cudaMemcpyAsync(c->d_slot_of_active, c->idx.slot_of_active.data(), c->idx.slot_of_active.size() * 4,
                       cudaMemcpyHostToDevice, c->stream),
       "copy slot map");
    if (!c->idx.tiles.empty())
        CK(cudaMemcpyAsync(c->d_tiles, c->idx.tiles.data(), c->idx.tiles.size() * 4, cudaMemcpyHostToDevice,
                           c->stream),
           "copy tile records");
    if (!c->idx.pair_items.empty())
        CK(cudaMemcpyAsync(c->d_items, c->idx.pair_items.data(), c->idx.pair_items.size() * 8,
                           cudaMemcpyHostToDevice, c->stream),
           "copy pair items");
    if (!c->idx.rest_chunks.empty())
        CK(cudaMemcpyAsync(c->d_rest, c->idx.rest_chunks.data(), c->idx.rest_chunks.size() * 8,
                           cudaMemcpyHostToDevice, c->stream),
           "copy rest chunks");
    // Padding slots are never read by the step kernel; zero both buffers so
    // that checkpoints and dumps are deterministic.
    CK(cudaMemsetAsync(c->f_raw[0], 0, raw_pop_bytes(c), c->stream), "clear f0");
    CK(cudaMemsetAsync(c->f_raw[1], 0, raw_pop_bytes(c), c->stream), "clear f1");
    CK(cudaMemsetAsync(c->d_status, 0, 4, c->stream), "clear status");
    CK(cudaStreamSynchronize(c->stream), "sync geometry upload");
    c->has_geom = true;
    c->has_state = false;
    c->cur = 0;
    c->t = 0;
    return LBM_OK;
}

}  // namespace lbm

extern "C" {

lbm_status lbm_fluid_count(lbm_ctx *c, int64_t *n) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (!n) return fail(c, LBM_ERR_ARG, "NULL output");
    *n = c->idx.n_active;
    return LBM_OK;
}

lbm_status lbm_params_check(const lbm_params *p, double *nu_out, double *omega_out, const char **why) {
    const char *msg = "";
    double nu = 0.0, omega = 0.0;
    lbm_status st = LBM_ERR_ARG;
    if (!p) {
        msg = "params is NULL";
    } else {
        nu = p->nu;
        if (!(nu > 0.0) && (!(p->Re > 0.0) || !(p->L_char > 0.0) || !(std::fabs(p->u_char) > 0.0))) {
            msg = "give nu > 0, or Re, u_char and L_char > 0";
        } else {
            if (!(nu > 0.0)) nu = std::fabs(p->u_char) * p->L_char / p->Re;  // Re = u L / nu (Sec. 2.2)
            omega = 1.0 / (3.0 * nu + 0.5);  // tau = nu / theta0 + 1/2 (Sec. 2.1)
            const double g[4] = {p->omega3, p->omega4, p->omega5, p->omega6};
            const double cs = 1.0 / std::sqrt(3.0);
            if (!(omega > 0.0 && omega < 2.0))
                msg = "omega outside (0, 2)";
            else if (!std::all_of(g, g + 4, [](double r) { return r > 0.0 && r < 2.0; }))
                msg = "ghost rates must lie in (0, 2)";
            else if (!(std::fabs(p->u_in) < cs) || !(std::fabs(p->u_char) < cs))
                msg = "velocities must stay below the lattice sound speed";
            else if (p->inlet_profile != LBM_PROFILE_PLUG && p->inlet_profile != LBM_PROFILE_PARABOLIC)
                msg = "unknown inlet profile";
            else if (!(p->noise_amp >= 0.0) || !(p->rho_out > 0.0))
                msg = "bad noise or rho_out";
            else if (p->inlet_ramp < 0)
                msg = "negative inlet ramp";
            else
                st = LBM_OK;
        }
    }
    if (nu_out) *nu_out = st == LBM_OK ? nu : 0.0;
    if (omega_out) *omega_out = st == LBM_OK ? omega : 0.0;
    if (why) *why = msg;
    return st;
}

lbm_status lbm_params_from_physical(const lbm_physical *ph, lbm_params *p, double out[5], const char **why) {
    const char *msg = "";
    lbm_status st = LBM_ERR_ARG;
    double lu[5] = {0, 0, 0, 0, 0};
    if (!ph || !p) {
        msg = "physical description or params is NULL";
    } else if (!(ph->Re > 0.0) || !(ph->d_thr > 0.0) || !(ph->rho > 0.0) || !(ph->mu > 0.0) || !(ph->delta_r > 0.0)) {
        msg = "Re, d_thr, rho, mu and delta_r must be > 0";
    } else if (!(ph->delta_t > 0.0) && !(ph->CFL > 0.0)) {
        msg = "give delta_t > 0 or CFL > 0";
    } else {
        // throat mean velocity from the throat Reynolds number Re = rho u_thr d_thr / mu (Sec. 2.2)
        const double u_thr = ph->mu * ph->Re / (ph->rho * ph->d_thr);
        // time step of the CFL rule CFL = 2 u_thr dt / dr (Sec. 2.2) when none is given
        const double dt = ph->delta_t > 0.0 ? ph->delta_t
                                            : ph->rho * ph->d_thr * ph->delta_r * ph->CFL / (2.0 * ph->mu * ph->Re);
        lu[0] = ph->d_thr / ph->delta_r;                          // L_char: throat diameter in cells
        lu[1] = u_thr * dt / ph->delta_r;                         // u_char: throat velocity in cells per step
        lu[2] = ph->mu * dt / (ph->rho * ph->delta_r * ph->delta_r);  // nu in lattice units
        lu[3] = 2.0 * lu[1];                                      // CFL of the throat mean velocity
        lu[4] = dt;
        lbm_params q = *p;
        q.nu = 0.0;  // derived from Re = u_char L_char / nu
        q.Re = ph->Re;
        q.u_char = lu[1];
        q.L_char = lu[0];
        st = lbm_params_check(&q, nullptr, nullptr, &msg);
        if (st == LBM_OK) *p = q;
    }
    if (out)
        for (int k = 0; k < 5; ++k) out[k] = st == LBM_OK ? lu[k] : 0.0;
    if (why) *why = msg;
    return st;
}

lbm_status lbm_set_params(lbm_ctx *c, const lbm_params *p) {
    if (!c) return LBM_ERR_ARG;
    double nu, omega;
    const char *why;
    if (lbm_params_check(p, &nu, &omega, &why) != LBM_OK) return fail(c, LBM_ERR_ARG, why);
    const double g[4] = {p->omega3, p->omega4, p->omega5, p->omega6};
    c->params = *p;
    c->params.nu = nu;
    if (!(c->params.d_in > 0.0)) c->params.d_in = c->desc.nx;
    if (c->params.axis_x < 0.0) c->params.axis_x = c->desc.nx / 2.0;
    if (c->params.axis_y < 0.0) c->params.axis_y = c->desc.ny / 2.0;
    c->omega = omega;
    c->ghost1 = g[0] == 1.0 && g[1] == 1.0 && g[2] == 1.0 && g[3] == 1.0;
    c->has_params = true;
    c->err.clear();
    return LBM_OK;
}

lbm_status lbm_get_omega(lbm_ctx *c, double *omega) {
    lbm_status st = need(c, false, true, false);
    if (st) return st;
    if (!omega) return fail(c, LBM_ERR_ARG, "NULL output");
    *omega = c->omega;
    return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx *c, double rho, const double u[3]) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (!u || !(rho > 0.0)) return fail(c, LBM_ERR_ARG, "need rho > 0 and u");
    DeviceGuard g(c->desc.device);
    c->cur = 0;
    CK(DISPATCH(c->desc.precision, launch_init_eq, c->f[0], c->d_slot_of_active, c->idx.n_active, c->idx.nslots,
                fp16_scale(c), nullptr, nullptr, rho, u[0], u[1], u[2], c->stream),
       "init equilibrium");
    st = reset_state(c);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream), "sync init");
    return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx *c, const double *rho, const double *u, int32_t layout) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (!rho || !u || (layout != LBM_LAYOUT_ACTIVE && layout != LBM_LAYOUT_BOX))
        return fail(c, LBM_ERR_ARG, "need rho, u and a valid layout");
    DeviceGuard g(c->desc.device);
    const int64_t n = c->idx.n_active;
    double *d = (double *)dev_alloc(c, (size_t)n * 4 * 8);
    if (!d) return fail(c, LBM_ERR_OOM, "staging allocation failed");
    cudaError_t e;
    if (layout == LBM_LAYOUT_ACTIVE) {  // the caller's arrays are already in the device's order: copy them as they are
        e = cudaMemcpyAsync(d, rho, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, u, (size_t)n * 3 * 8, cudaMemcpyHostToDevice, c->stream);
    } else {
        std::vector<double> h((size_t)n * 4);
        for_active(c, layout, [&](int64_t k, int64_t r) {
            h[(size_t)k] = rho[r];
            for (int a = 0; a < 3; ++a) h[(size_t)n + 3 * (size_t)k + a] = u[3 * r + a];
        });
        e = cudaMemcpyAsync(d, h.data(), (size_t)n * 4 * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // h leaves scope
    }
    c->cur = 0;
    if (e == cudaSuccess)
        e = DISPATCH(c->desc.precision, launch_init_eq, c->f[0], c->d_slot_of_active, n, c->idx.nslots,
                     fp16_scale(c), d, d + n, 1.0, 0.0, 0.0, 0.0, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, d, (size_t)n * 4 * 8);
    if (e != cudaSuccess) return cuda_fail(c, e, "init fields");
    return reset_state(c);
}

lbm_status lbm_set_populations(lbm_ctx *c, const double *f, int32_t layout) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (!f || (layout != LBM_LAYOUT_ACTIVE && layout != LBM_LAYOUT_BOX))
        return fail(c, LBM_ERR_ARG, "need f and a valid layout");
    DeviceGuard g(c->desc.device);
    const int64_t n = c->idx.n_active;
    const size_t bytes = (size_t)n * 27 * 8;
    double *d = (double *)dev_alloc(c, bytes);
    if (!d) return fail(c, LBM_ERR_OOM, "staging allocation failed");
    cudaError_t e = cudaSuccess;
    if (layout == LBM_LAYOUT_ACTIVE) {
        e = cudaMemcpyAsync(d, f, bytes, cudaMemcpyHostToDevice, c->stream);
    } else {
        std::vector<double> h((size_t)n * 27);
        for_active(c, layout, [&](int64_t k, int64_t r) { memcpy(&h[27 * (size_t)k], f + 27 * r, 27 * 8); });
        e = cudaMemcpyAsync(d, h.data(), bytes, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    c->cur = 0;
    if (e == cudaSuccess)
        e = DISPATCH(c->desc.precision, launch_set_populations, c->f[0], c->d_slot_of_active, n, c->idx.nslots,
                     fp16_scale(c), d, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, d, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "set populations");
    return reset_state(c);
}

lbm_status lbm_get_populations(lbm_ctx *c, double *f, int32_t layout) {
    lbm_status st = need(c, true, false, true);
    if (st) return st;
    if (!f || (layout != LBM_LAYOUT_ACTIVE && layout != LBM_LAYOUT_BOX))
        return fail(c, LBM_ERR_ARG, "need f and a valid layout");
    DeviceGuard g(c->desc.device);
    const int64_t n = c->idx.n_active;
    const size_t bytes = (size_t)n * 27 * 8;
    double *d = (double *)dev_alloc(c, bytes);
    if (!d) return fail(c, LBM_ERR_OOM, "staging allocation failed");
    cudaError_t e = DISPATCH(c->desc.precision, launch_get_populations, c->f[c->cur], c->d_slot_of_active, n,
                             c->idx.nslots, 1.0f / fp16_scale(c), d, c->stream);
    if (layout == LBM_LAYOUT_ACTIVE) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    } else {
        std::vector<double> h((size_t)n * 27);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) {
            memset(f, 0, (size_t)layout_count(c, layout) * 27 * 8);
            for_active(c, layout, [&](int64_t k, int64_t r) { memcpy(f + 27 * r, &h[27 * (size_t)k], 27 * 8); });
        }
    }
    dev_free(c, d, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "get populations");
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, int64_t n) {
    const TraceRange trace("lbm_step");
    lbm_status st = need(c, true, true, true);
    if (st) return st;
    if (n < 0) return fail(c, LBM_ERR_ARG, "negative step count");
    DeviceGuard g(c->desc.device);
    StepArgs a{};
    lbm::ctx_step_args(c, &a);
    for (int64_t k = 0; k < n; ++k) {
        const int64_t t_new = c->t + 1;
        a.fin = c->f[c->cur];
        a.fout = c->f[1 - c->cur];
        a.t_new = t_new;
        a.flags = 0;
        const bool check = c->check_every > 0 && t_new % c->check_every == 0;
        if (check) a.flags |= STEP_REDUCE;
        if (c->stats_on && t_new >= c->stats_start && (t_new - c->stats_start) % c->stats_stride == 0) {
            a.flags |= STEP_STATS | (c->stats_ncomp == STATS_FULL ? STEP_STATS_FULL : 0);
            ++c->stats_samples;
        }
        int launched = 0;
        CK(DISPATCH(c->desc.precision, launch_step, a, c->ghost1, c->stream, &launched, &c->side), "step kernel");
        c->kernel_launches += launched;
        if (check) {
            CK(launch_finalize(c->d_partials, step_partials(c), c->d_health, c->d_status, c->stream), "finalize");
            ++c->kernel_launches;
        }
        c->cur = 1 - c->cur;
        c->t = t_new;
    }
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx *c) {
    const TraceRange trace("lbm_sync");
    if (!c) return LBM_ERR_ARG;
    DeviceGuard g(c->desc.device);
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (!c->has_geom) return LBM_OK;
    uint32_t status = 0;
    CK(cudaMemcpyAsync(&status, c->d_status, 4, cudaMemcpyDeviceToHost, c->stream), "read status");
    CK(cudaStreamSynchronize(c->stream), "sync status");
    if (c->check_every > 0) {
        CK(cudaMemcpyAsync(c->health, c->d_health, 6 * 8, cudaMemcpyDeviceToHost, c->stream), "read health");
        CK(cudaStreamSynchronize(c->stream), "sync health");
    }
    if (status & 2u) return fail(c, LBM_ERR_TIMEOUT, "a bounded device-side wait gave up (step kernel)");
    if (status & 1u) return fail(c, LBM_ERR_UNSTABLE, "a health check found non-finite populations");
    return LBM_OK;
}

lbm_status lbm_step_count(lbm_ctx *c, int64_t *t) {
    if (!c || !t) return LBM_ERR_ARG;
    *t = c->t;
    return LBM_OK;
}

lbm_status lbm_set_check_every(lbm_ctx *c, int64_t k) {
    if (!c) return LBM_ERR_ARG;
    if (k < 0) return fail(c, LBM_ERR_ARG, "negative check interval");
    c->check_every = k;
    return LBM_OK;
}

lbm_status lbm_get_moments(lbm_ctx *c, double *rho, double *u, int32_t layout) {
    const TraceRange trace("lbm_get_moments");
    lbm_status st = need(c, true, false, true);
    if (st) return st;
    if ((!rho && !u) || (layout != LBM_LAYOUT_ACTIVE && layout != LBM_LAYOUT_BOX))
        return fail(c, LBM_ERR_ARG, "need an output array and a valid layout");
    DeviceGuard g(c->desc.device);
    const int64_t n = c->idx.n_active;
    const size_t bytes = (size_t)n * 4 * 8;
    if (layout == LBM_LAYOUT_ACTIVE) {
        // split on the device, then one copy straight into each of the caller's arrays
        double *d = (double *)dev_alloc(c, 2 * bytes);
        if (!d) return fail(c, LBM_ERR_OOM, "staging allocation failed");
        double *dr = d + 4 * n, *du = d + 5 * n;
        cudaError_t e = DISPATCH(c->desc.precision, launch_moments, c->f[c->cur], c->d_slot_of_active, n,
                                 c->idx.nslots, 1.0f / fp16_scale(c), d, c->stream);
        if (e == cudaSuccess) e = launch_split_moments(d, n, dr, du, c->stream);
        if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, dr, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, (size_t)n * 3 * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, d, 2 * bytes);
        if (e != cudaSuccess) return cuda_fail(c, e, "get moments");
        return LBM_OK;
    }
    double *d = (double *)dev_alloc(c, bytes);
    if (!d) return fail(c, LBM_ERR_OOM, "staging allocation failed");
    std::vector<double> h((size_t)n * 4);
    cudaError_t e = DISPATCH(c->desc.precision, launch_moments, c->f[c->cur], c->d_slot_of_active, n, c->idx.nslots,
                             1.0f / fp16_scale(c), d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, d, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "get moments");
    const int64_t total = layout_count(c, layout);
    if (rho) memset(rho, 0, (size_t)total * 8);
    if (u) memset(u, 0, (size_t)total * 3 * 8);
    for_active(c, layout, [&](int64_t k, int64_t r) {
        if (rho) rho[r] = h[4 * (size_t)k];
        if (u)
            for (int a = 0; a < 3; ++a) u[3 * r + a] = h[4 * (size_t)k + 1 + a];
    });
    return LBM_OK;
}

lbm_status lbm_get_totals(lbm_ctx *c, double *mass, double mom[3]) {
    const TraceRange trace("lbm_get_totals");
    lbm_status st = need(c, true, false, true);
    if (st) return st;
    DeviceGuard g(c->desc.device);
    CK(DISPATCH(c->desc.precision, launch_reduce, c->f[c->cur], c->d_slot_of_active, c->idx.n_active, c->idx.nslots,
                1.0f / fp16_scale(c), c->d_partials, c->stream),
       "reduce");
    CK(launch_finalize(c->d_partials, node_blocks(c->idx.n_active), c->d_health, c->d_status, c->stream), "finalize");
    CK(cudaMemcpyAsync(c->health, c->d_health, 6 * 8, cudaMemcpyDeviceToHost, c->stream), "read totals");
    CK(cudaStreamSynchronize(c->stream), "sync totals");
    if (mass) *mass = c->health[0];
    if (mom)
        for (int a = 0; a < 3; ++a) mom[a] = c->health[1 + a];
    return LBM_OK;
}

lbm_status lbm_get_health(lbm_ctx *c, double out[6]) {
    if (!c || !out) return LBM_ERR_ARG;
    for (int k = 0; k < 6; ++k) out[k] = c->health[k];
    return LBM_OK;
}

// (Re)allocate the accumulators with the row count of the current mode.
lbm_status stats_alloc(lbm_ctx *c) {
    const int want = c->stats_mode == LBM_STATS_FULL ? STATS_FULL : STATS_AXIAL;
    if (c->d_stats && c->stats_ncomp == want) return LBM_OK;
    dev_free(c, c->d_stats, stats_bytes(c));
    c->d_stats = nullptr;
    c->stats_ncomp = 0;
    c->stats_samples = 0;
    const size_t bytes = (size_t)want * (size_t)c->idx.nslots * 8;
    c->d_stats = (double *)dev_alloc(c, bytes);
    if (!c->d_stats) return fail(c, LBM_ERR_OOM, "statistics allocation failed");
    c->stats_ncomp = want;
    CK(cudaMemsetAsync(c->d_stats, 0, bytes, c->stream), "clear stats");
    return LBM_OK;
}

lbm_status lbm_stats_set_mode(lbm_ctx *c, int32_t mode) {
    if (!c) return LBM_ERR_ARG;
    if (mode != LBM_STATS_AXIAL && mode != LBM_STATS_FULL) return fail(c, LBM_ERR_ARG, "unknown statistics mode");
    if (c->stats_on && mode != c->stats_mode) return fail(c, LBM_ERR_STATE, "statistics are being sampled");
    c->stats_mode = mode;
    c->err.clear();
    return LBM_OK;
}

lbm_status lbm_stats_begin(lbm_ctx *c, int64_t stride) {
    lbm_status st = need(c, true, false, true);
    if (st) return st;
    if (stride < 1) return fail(c, LBM_ERR_ARG, "stride must be >= 1");
    DeviceGuard g(c->desc.device);
    st = stats_alloc(c);
    if (st) return st;
    c->stats_on = true;
    c->stats_stride = stride;
    c->stats_start = c->t + 1;
    return LBM_OK;
}

lbm_status lbm_stats_end(lbm_ctx *c) {
    if (!c) return LBM_ERR_ARG;
    c->stats_on = false;
    return LBM_OK;
}

lbm_status lbm_stats_reset(lbm_ctx *c) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    DeviceGuard g(c->desc.device);
    if (c->d_stats) CK(cudaMemsetAsync(c->d_stats, 0, stats_bytes(c), c->stream), "clear stats");
    c->stats_samples = 0;
    return LBM_OK;
}

// Means of the first ncomp accumulator rows, per active cell, to the host
// ([n_active][ncomp]).
lbm_status stats_means(lbm_ctx *c, int ncomp, std::vector<double> &h) {
    const int64_t n = c->idx.n_active;
    const size_t bytes = (size_t)n * ncomp * 8;
    h.assign((size_t)n * ncomp, 0.0);
    if (n == 0) return LBM_OK;
    double *d = (double *)dev_alloc(c, bytes);
    if (!d) return fail(c, LBM_ERR_OOM, "staging allocation failed");
    cudaError_t e = launch_stats_mean(c->d_stats, ncomp, c->d_slot_of_active, n, c->idx.nslots,
                                      1.0 / (double)c->stats_samples, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, d, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "stats readback");
    return LBM_OK;
}

lbm_status lbm_stats_get(lbm_ctx *c, double *mean_uz, double *mean_uzuz, int64_t *n_samples, int32_t layout) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (layout != LBM_LAYOUT_ACTIVE && layout != LBM_LAYOUT_BOX) return fail(c, LBM_ERR_ARG, "bad layout");
    if (n_samples) *n_samples = c->stats_samples;
    if (!mean_uz && !mean_uzuz) return LBM_OK;
    const int64_t total = layout_count(c, layout);
    if (mean_uz) memset(mean_uz, 0, (size_t)total * 8);
    if (mean_uzuz) memset(mean_uzuz, 0, (size_t)total * 8);
    if (!c->d_stats || c->stats_samples == 0) return LBM_OK;
    DeviceGuard g(c->desc.device);
    std::vector<double> h;
    st = stats_means(c, STATS_AXIAL, h);
    if (st) return st;
    for_active(c, layout, [&](int64_t k, int64_t r) {
        if (mean_uz) mean_uz[r] = h[2 * (size_t)k];
        if (mean_uzuz) mean_uzuz[r] = h[2 * (size_t)k + 1];
    });
    return LBM_OK;
}

lbm_status lbm_stats_get_full(lbm_ctx *c, double *mean, int64_t *n_samples, int32_t layout) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (layout != LBM_LAYOUT_ACTIVE && layout != LBM_LAYOUT_BOX) return fail(c, LBM_ERR_ARG, "bad layout");
    if (n_samples) *n_samples = c->stats_samples;
    if (!mean) return LBM_OK;
    if (c->stats_ncomp != STATS_FULL && c->stats_samples > 0)
        return fail(c, LBM_ERR_STATE, "the accumulators hold axial statistics only");
    const int64_t total = layout_count(c, layout);
    memset(mean, 0, (size_t)total * LBM_STATS_FULL_COMPONENTS * 8);
    if (!c->d_stats || c->stats_samples == 0) return LBM_OK;
    DeviceGuard g(c->desc.device);
    std::vector<double> h;
    st = stats_means(c, STATS_FULL, h);
    if (st) return st;
    for_active(c, layout, [&](int64_t k, int64_t r) {
        for (int q = 0; q < LBM_STATS_FULL_COMPONENTS; ++q)
            mean[(size_t)r * LBM_STATS_FULL_COMPONENTS + q] = h[(size_t)k * STATS_FULL + STATS_AXIAL + q];
    });
    return LBM_OK;
}

// Checkpoint image: header, then the current population buffer (native
// storage, bitwise), then the statistics accumulators if allocated
// (has_stats holds their row count: 0, 2 or 18).
struct CkptHeader {
    uint64_t magic;
    int32_t version, precision, nx, ny, nz, periodic;
    float scale;
    int32_t has_stats;
    int64_t nslots, n_active, t, stats_samples, stats_stride, stats_start;
    int32_t stats_on, reserved;
};
static const uint64_t CKPT_MAGIC = 0x4c424d3237434b50ULL;  // "LBM27CKP"
static const int32_t CKPT_VERSION = 2;

lbm_status lbm_checkpoint_size(lbm_ctx *c, size_t *bytes) {
    lbm_status st = need(c, true, false, true);
    if (st) return st;
    if (!bytes) return fail(c, LBM_ERR_ARG, "NULL output");
    *bytes = sizeof(CkptHeader) + pop_bytes(c) + stats_bytes(c);
    return LBM_OK;
}

lbm_status lbm_checkpoint(lbm_ctx *c, void *buf, size_t bytes) {
    size_t need_bytes = 0;
    lbm_status st = lbm_checkpoint_size(c, &need_bytes);
    if (st) return st;
    if (!buf || bytes < need_bytes) return fail(c, LBM_ERR_ARG, "checkpoint buffer too small");
    DeviceGuard g(c->desc.device);
    CkptHeader h{};
    h.magic = CKPT_MAGIC;
    h.version = CKPT_VERSION;
    h.precision = c->desc.precision;
    h.nx = c->desc.nx;
    h.ny = c->desc.ny;
    h.nz = c->desc.nz;
    h.periodic = c->desc.periodic;
    h.scale = fp16_scale(c);
    h.has_stats = c->d_stats ? c->stats_ncomp : 0;
    h.nslots = c->idx.nslots;
    h.n_active = c->idx.n_active;
    h.t = c->t;
    h.stats_samples = c->stats_samples;
    h.stats_stride = c->stats_stride;
    h.stats_start = c->stats_start;
    h.stats_on = c->stats_on;
    char *p = static_cast<char *>(buf);
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    CK(cudaMemcpyAsync(p, c->f[c->cur], pop_bytes(c), cudaMemcpyDeviceToHost, c->stream), "checkpoint f");
    p += pop_bytes(c);
    if (c->d_stats)
        CK(cudaMemcpyAsync(p, c->d_stats, stats_bytes(c), cudaMemcpyDeviceToHost, c->stream), "checkpoint stats");
    CK(cudaStreamSynchronize(c->stream), "sync checkpoint");
    return LBM_OK;
}

lbm_status lbm_restore(lbm_ctx *c, const void *buf, size_t bytes) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (!buf || bytes < sizeof(CkptHeader)) return fail(c, LBM_ERR_ARG, "checkpoint too small");
    CkptHeader h;
    memcpy(&h, buf, sizeof h);
    if (h.magic != CKPT_MAGIC || h.version != CKPT_VERSION) return fail(c, LBM_ERR_ARG, "not a checkpoint image");
    if (h.has_stats != 0 && h.has_stats != STATS_AXIAL && h.has_stats != STATS_FULL)
        return fail(c, LBM_ERR_ARG, "checkpoint statistics block is malformed");
    if (h.precision != c->desc.precision || h.nx != c->desc.nx || h.ny != c->desc.ny || h.nz != c->desc.nz ||
        h.periodic != c->desc.periodic || h.scale != fp16_scale(c) || h.nslots != c->idx.nslots ||
        h.n_active != c->idx.n_active)
        return fail(c, LBM_ERR_ARG, "checkpoint does not match this context's geometry or precision");
    const size_t need_bytes = sizeof h + pop_bytes(c) + (size_t)h.has_stats * (size_t)h.nslots * 8;
    if (bytes < need_bytes) return fail(c, LBM_ERR_ARG, "checkpoint truncated");
    DeviceGuard g(c->desc.device);
    const char *p = static_cast<const char *>(buf) + sizeof h;
    c->cur = 0;
    CK(cudaMemcpyAsync(c->f[0], p, pop_bytes(c), cudaMemcpyHostToDevice, c->stream), "restore f");
    p += pop_bytes(c);
    if (h.has_stats) {
        c->stats_on = false;
        c->stats_mode = h.has_stats == STATS_FULL ? LBM_STATS_FULL : LBM_STATS_AXIAL;
        st = stats_alloc(c);
        if (st) return st;
        CK(cudaMemcpyAsync(c->d_stats, p, stats_bytes(c), cudaMemcpyHostToDevice, c->stream), "restore stats");
    }
    CK(cudaMemsetAsync(c->d_status, 0, 4, c->stream), "reset status");
    CK(cudaStreamSynchronize(c->stream), "sync restore");
    c->t = h.t;
    c->stats_samples = h.stats_samples;
    c->stats_stride = h.stats_stride;
    c->stats_start = h.stats_start;
    c->stats_on = h.stats_on != 0 && h.has_stats;
    c->has_state = true;
    return LBM_OK;
}

lbm_status lbm_layout_info(lbm_ctx *c, int64_t *slots, int64_t *buffer_bytes, int64_t *device_bytes) {
    lbm_status st = need(c, true, false, false);
    if (st) return st;
    if (slots) *slots = c->idx.nslots;
    if (buffer_bytes) *buffer_bytes = (int64_t)pop_bytes(c);
    if (device_bytes) *device_bytes = c->device_bytes;
    return LBM_OK;
}

lbm_status lbm_kernel_launches(lbm_ctx *c, int64_t *n) {
    if (!c || !n) return LBM_ERR_ARG;
    *n = c->kernel_launches;
    return LBM_OK;
}

}  // extern "C"
