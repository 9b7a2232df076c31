// Internal declarations of the GB300 lattice Boltzmann library: device
// argument blocks, the context, and the per-precision kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// NVTX range over a host call (a no-op unless a profiler is attached): the
// step loop, the reductions, index building and the server's ticks show up
// by name on an Nsight timeline.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Cells per work chunk: a chunk is CHUNK consecutive x positions of one row
// (fixed y, z).  Every row's storage starts and ends on a CHUNK boundary so
// that chunk lanes map to consecutive, aligned storage slots.
constexpr int CHUNK = 8;
#ifndef LBM_STEP_THREADS
#define LBM_STEP_THREADS 128
#endif
constexpr int STEP_THREADS = LBM_STEP_THREADS;
constexpr int REDUCE_SLOTS = 8;  // doubles per block partial

// Per-slot link word.
//   bits 0..26 : link i is a wall link: the pull source x - c_i is solid or
//                outside a non-periodic face.  The cell then writes its
//                reflected population f*_{26-i} into the ghost slot that
//                stands at x - c_i in population array i, so that the next
//                step's pull of population i is the halfway bounce-back.
//                At a padding / ghost slot, bit i instead marks population
//                array i as read there (a wall link's ghost value or a
//                periodic copy); the other arrays take filler.
//   bits 27..28: node type (0 fluid, 1 inlet, 2 outlet, 3 padding / ghost)
//   bits 29..31: inlet/outlet partner direction (0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z)
enum : uint32_t {
    LINK_MASK = (1u << 27) - 1u,
    TYPE_SHIFT = 27,
    TYPE_FLUID = 0,
    TYPE_INLET = 1,
    TYPE_OUTLET = 2,
    TYPE_PAD = 3,
    DIR_SHIFT = 29,
};

enum : int { STEP_REDUCE = 1, STEP_STATS = 2, STEP_STATS_FULL = 4 };

// Statistics accumulators, [components][slots] doubles: 0 sum u_z, 1 sum u_z^2
// (always), and with full statistics 2..4 sum u, 5..10 sum u_a u_b
// (xx, yy, zz, xy, xz, yz), 11..16 sum sigma_ab (same order), 17 sum rho.
constexpr int STATS_AXIAL = 2;
constexpr int STATS_FULL = 18;

// Chunk records (int2): x = row, y = x0 | fluid-lane mask << CHUNK_LANES_SHIFT.
// The lane mask lets the gather start without waiting for the per-cell link
// words.  Inlet/outlet nodes are not in chunks: a separate boundary-node list
// (int4: x, row, slot, link word) drives the boundary kernel.
enum : uint32_t {
    CHUNK_X0_MASK = (1u << 20) - 1u,
    CHUNK_LANES_SHIFT = 20,
};

// Row records: rows run along the row axis (x, or z for lattices longer in z
// than in x).  In storage coordinates p (along the row) and a, b (across it),
// (p, a, b) = (x, y, z) for rows along x and (z, x, y) for rows along z, and
// rows are indexed over the box extended by one ghost layer in a and b,
// row = (a + 1) + (n_a + 2) (b + 1).  Each row record holds the storage
// bases of the nine neighbour rows (a - ca, b - cb), j = (ca + 1) + 3 (cb + 1),
// so that the slot of the pull source of population i of the cell at p is
// nb[j] + p - cp for every link (j = 4 is the row itself).
constexpr int ROW_RECORD_INTS = 12;

// Tile records of the tile fluid kernel: a tile is up to four consecutive
// chunks of one row, i.e. up to 32 consecutive positions [p0, p0 + 32).  A
// record holds p0 (with the fast flag TILE_FAST: 32 fluid cells, none with
// a wall link or a wrap-around copy), the fluid-lane mask (bit l: position
// p0 + l is a fluid cell), the present-lane mask (bit l: p0 + l lies in one
// of the tile's chunks; other lanes store nothing) and the row's nine
// neighbour bases (as in the row record), so that a tile needs no dependent
// index load.
constexpr int TILE_INTS = 12;
constexpr uint32_t TILE_FAST = 1u << 31;

// Group a chunk list (in row order) into tile records, in the same order;
// mask: the link words, n_row / periodic_row: the row axis (wrap-around
// copies at its ends).
std::vector<int32_t> build_tiles(const std::vector<int2> &chunks, const std::vector<int32_t> &row_nb,
                                 const std::vector<uint32_t> &mask, int n_row, bool periodic_row);
// Work items of the FP16S pair kernel over tile records in row order: (t, t + 1)
// for two consecutive fast tiles, taken greedily from the start.
std::vector<int2> build_pair_items(const std::vector<int32_t> &tiles);
// The chunks of every tile that is in no pair item, in order: the chunk
// kernel's list beside the pair kernel.
std::vector<int2> build_rest_chunks(const std::vector<int2> &chunks, const std::vector<int32_t> &tiles,
                                    const std::vector<int2> &pairs);

// Fluid kernel of the FP32 / FP16S steps: AUTO is the tile kernel in FP32
// and the chunk kernel in FP16S; the others are kept for testing.
enum class FluidKernel { AUTO, CHUNK, TILE, PAIRS };

// A second stream and its fork / join events: a step's wall-cell and
// inlet/outlet kernels run on it beside the fluid kernel.  They read the
// same input buffer and write other slots and other partial sums.
struct SideStream {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Flow parameters in the arithmetic precision of a kernel.
template <class R>
struct FlowParams {
    R omega;
    R ghost[4];
    R u_in, d_in, axis_x, axis_y, noise_amp, rho_out;
};

struct alignas(16) StepArgs {
    const void *fin;        // population arrays [27][stride], storage type of the kernel
    void *fout;
    const uint32_t *mask;
    const int4 *row_nb;     // [rows][3] row records
    const int2 *chunks;     // chunk records (fluid cells)
    int32_t nchunks;
    const int4 *bnodes;     // boundary nodes (x, row, slot, link word)
    int32_t nbnodes;
    int32_t fluid_blocks;   // blocks of the fluid kernel (offset of the boundary kernel's partials)
    uint32_t *status;       // bit 1: a bounded device wait gave up
    int32_t nx, ny, nz;     // box (physical x, y, z)
    int32_t na_e;           // extended extent of the first cross axis (decodes a row index)
    int32_t n_row;          // cells along the row axis
    int32_t row_axis;       // 0: rows along x, 2: rows along z
    int32_t flags;          // STEP_REDUCE | STEP_STATS
    int32_t profile;
    int32_t periodic_row;   // the row axis is periodic (wrap-around copies at p = -1 and n_row)
    FlowParams<double> pd;
    FlowParams<float> pf;
    uint64_t seed;
    int64_t t_new;
    float scale, inv_scale;
    int64_t stride;         // elements between two population arrays (= slot count)
    double *stats;          // [STATS_AXIAL or STATS_FULL][stride] accumulators
    double *partials;       // [gridDim.x][REDUCE_SLOTS]
    int32_t prefetch_ahead; // fluid blocks between a block and the one whose sources it prefetches to L2 (0: off)
    int32_t inlet_ramp;     // steps over which the inlet velocity rises from 0 (0: impulsive start)
    const int32_t *wall_qidx;  // per slot: wall-distance record of the cell, or -1 (NULL: q = 1/2 everywhere)
    const uint8_t *wall_q;     // records of 32 bytes: q = k / 256 of wall link i in byte i
    const int4 *wnodes;        // cells with interpolated walls (x, row, slot, record), out of the chunk lanes
    int32_t nwnodes;
    int32_t wide_offsets;      // 1: 64-bit element offsets even when 32 bits would do (LBM_WIDE_OFFSETS=1)
    const int32_t *tiles;      // tile records of the tile fluid kernels (NULL: chunk kernel)
    int32_t ntiles;
    const int2 *items;         // FP16S pairs of fast tiles (NULL: tile kernel); chunks then holds the rest
    int32_t nitems;
};

// Launchers, one set per storage precision (P = 0 FP64, 1 FP32, 2 FP16S).
// Offsets into a population buffer fit in 32 bits (unsigned) when
// 27 * slots < 2^32; larger lattices use 64-bit offsets.
constexpr int64_t MAX_SLOTS_32 = (int64_t)0xFFFFFFFFu / 27 - 64;

template <int P>
cudaError_t launch_step(const StepArgs &a, bool ghost1, cudaStream_t s, int *launches = nullptr,
                        const SideStream *side = nullptr);
// L2 prefetch lookahead of the fluid kernel in blocks: a fixed share of the
// blocks resident on the device at once (occupancy x SM count); 0 = off.
template <int P>
int step_prefetch_ahead(bool ghost1, bool wide, int device);
// Blocks of one step's fluid kernel (partial-sum slots it writes).
template <int P>
int step_fluid_blocks(int32_t nchunks);
// Blocks of the tile fluid kernel (one warp per tile or per pair-kernel item)
// and of a grid with 16 threads per tile.
__host__ __device__ inline int tile_blocks(int64_t ntiles) {
    return (int)((ntiles + STEP_THREADS / 32 - 1) / (STEP_THREADS / 32));
}
__host__ __device__ inline int pair_blocks(int64_t nfast) { return (int)((nfast * 16 + STEP_THREADS - 1) / STEP_THREADS); }
template <int P>
cudaError_t launch_reduce(const void *f, const int32_t *slot_of_active, int64_t n, int64_t stride, float inv_scale,
                          double *partials, cudaStream_t s);
// Write the bounce-back ghost slots and periodic-x copies of buffer f from
// its active cells (after any host-side change of the state).
template <int P>
cudaError_t launch_fill_ghosts(void *f, const uint32_t *mask, const int2 *chunks, const int4 *row_nb,
                               int32_t nchunks, const int4 *bnodes, int32_t nbnodes, int64_t stride, int32_t n_row,
                               int32_t periodic_row, int32_t row_axis, cudaStream_t s);
template <int P>
cudaError_t launch_moments(const void *f, const int32_t *slot_of_active, int64_t n, int64_t stride,
                           float inv_scale, double *out4, cudaStream_t s);
template <int P>
cudaError_t launch_get_populations(const void *f, const int32_t *slot_of_active, int64_t n,
                                   int64_t stride, float inv_scale, double *out27, cudaStream_t s);
template <int P>
cudaError_t launch_set_populations(void *f, const int32_t *slot_of_active, int64_t n, int64_t stride,
                                   float scale, const double *in27, cudaStream_t s);
template <int P>
cudaError_t launch_init_eq(void *f, const int32_t *slot_of_active, int64_t n, int64_t stride,
                           float scale, const double *rho, const double *u, double rho0,
                           double ux, double uy, double uz, cudaStream_t s);

int fluid_blocks(int32_t nchunks);
int node_blocks(int64_t n);
cudaError_t launch_finalize(const double *partials, int nblocks, double *health, uint32_t *status,
                            cudaStream_t s);
cudaError_t launch_stats_mean(const double *stats, int ncomp, const int32_t *slot_of_active, int64_t n,
                              int64_t stride, double inv_n, double *out, cudaStream_t s);

// Host-side sparse index (built by geometry.cpp).
struct HostIndex {
    int64_t n_active = 0;
    int64_t nslots = 0;
    int64_t n_ghost = 0;                  // bounce-back ghost slots
    int32_t row_axis = 0;                 // 0: rows along x, 2: rows along z
    int32_t n_row = 0;                    // cells along the row axis
    int32_t na_e = 0, nb_e = 0;           // extended extents of the two cross axes (row grid)
    std::vector<int32_t> row_nb;          // [rows][ROW_RECORD_INTS]
    std::vector<int2> chunks;             // chunk records (fluid cells)
    std::vector<int32_t> tiles;           // [tiles][TILE_INTS] records of the tile fluid kernels
    std::vector<int2> pair_items;         // pairs of fast tiles, for the FP16S pair kernel
    std::vector<int2> rest_chunks;        // chunks of the other tiles, for the chunk kernel beside it
    std::vector<int4> bnodes;             // inlet/outlet nodes: x, row, slot, link word
    std::vector<uint32_t> mask;           // [nslots]
    std::vector<int32_t> slot_of_active;  // [n_active], active order = increasing box index
    std::vector<int64_t> box_of_active;   // [n_active]
};

// Slack (elements) allocated before and after every population buffer and
// around the link-word array (keeps 256-byte alignment of the buffers).
inline int64_t buffer_margin(int nx) { return ((int64_t)nx + 64 + 63) & ~(int64_t)63; }
constexpr int64_t MASK_MARGIN = 64;

// Returns "" on success, else a description of the inconsistency.  With
// max_slots > 0, a lattice needing more storage slots is refused before its
// per-slot arrays are allocated.  row_axis: LBM_ROWS_AUTO / X / Z.
std::string build_index(const uint8_t *flags, int nx, int ny, int nz, int periodic, HostIndex &out,
                        int64_t max_slots = 0, int row_axis = LBM_ROWS_AUTO);
// Row axis (0: x, 2: z) of a box for a requested LBM_ROWS_* value: AUTO takes
// z when the box is longer in z than in x.
int choose_row_axis(int nx, int ny, int nz, int requested);
// Independent check of the index invariants the kernels rely on ("" if all hold).
std::string validate_index(const HostIndex &ix, const uint8_t *flags, int nx, int ny, int nz, int periodic);

// Hooks into a context for the request server (implemented in api.cu).
int64_t ctx_footprint(const lbm_desc &desc, const HostIndex &ix);  // device bytes lbm_set_geometry allocates
lbm_status ctx_install_index(lbm_ctx *c, HostIndex &&idx);        // allocate + upload a built index
void ctx_step_args(lbm_ctx *c, StepArgs *out);                      // arguments of the next step
void ctx_advance(lbm_ctx *c, int64_t steps);                        // account for steps run elsewhere
int64_t ctx_steps(const lbm_ctx *c);
int64_t ctx_device_bytes(const lbm_ctx *c);
bool ctx_ready(const lbm_ctx *c);
bool ctx_ghost1(const lbm_ctx *c);
int ctx_precision(const lbm_ctx *c);
int64_t ctx_slots(const lbm_ctx *c);

}  // namespace lbm
