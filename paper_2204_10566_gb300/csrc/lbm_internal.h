// Internal declarations of the GB300 lattice Boltzmann library: device
// argument blocks, the context, and the per-precision kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

// Cells per work chunk: a chunk is CHUNK consecutive x positions of one row
// (fixed y, z).  Every row's storage starts and ends on a CHUNK boundary so
// that chunk lanes map to consecutive, aligned storage slots.
constexpr int CHUNK = 8;
constexpr int STEP_THREADS = 256;
constexpr int REDUCE_SLOTS = 8;  // doubles per block partial

// Per-slot link word.
//   bits 0..26 : population i must bounce back (its pull source x - c_i is a
//                wall or outside a non-periodic face)
//   bits 27..28: node type (0 fluid, 1 inlet, 2 outlet, 3 padding)
//   bits 29..31: inlet/outlet partner direction (0 +x, 1 -x, 2 +y, 3 -y, 4 +z, 5 -z)
enum : uint32_t {
    TYPE_SHIFT = 27,
    TYPE_FLUID = 0,
    TYPE_INLET = 1,
    TYPE_OUTLET = 2,
    TYPE_PAD = 3,
    DIR_SHIFT = 29,
};

enum : int { STEP_REDUCE = 1, STEP_STATS = 2 };

struct StepArgs {
    const void *fin;
    void *fout;
    const uint32_t *mask;
    const int32_t *row_base;
    const int2 *chunks;  // (row = y + ny z, x0)
    int64_t stride;      // elements between two populations (= slot count)
    int32_t nchunks;
    int32_t nx, ny, nz;
    int32_t flags;       // STEP_REDUCE | STEP_STATS
    int32_t profile;
    double omega;
    double ghost[4];
    double u_in, d_in, axis_x, axis_y, noise_amp, rho_out;
    uint64_t seed;
    int64_t t_new;
    float scale, inv_scale;
    double *stats;       // [2][stride]: sum u_z, sum u_z^2
    double *partials;    // [gridDim.x][REDUCE_SLOTS]
};

// Launchers, one set per storage precision (P = 0 FP64, 1 FP32, 2 FP16S).
template <int P>
cudaError_t launch_step(const StepArgs &a, bool ghost1, cudaStream_t s);
template <int P>
cudaError_t launch_reduce(const void *f, const uint32_t *mask, const int2 *chunks,
                          const int32_t *row_base, int32_t nchunks, int64_t stride, float inv_scale,
                          double *partials, cudaStream_t s);
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

int reduce_blocks(int32_t nchunks);
cudaError_t launch_finalize(const double *partials, int nblocks, double *health, uint32_t *status,
                            cudaStream_t s);
cudaError_t launch_stats_mean(const double *stats, const int32_t *slot_of_active, int64_t n,
                              int64_t stride, double inv_n, double *out2, cudaStream_t s);

// Host-side sparse index (built by geometry.cpp).
struct HostIndex {
    int64_t n_active = 0;
    int64_t nslots = 0;
    std::vector<int32_t> row_base;        // [ny*nz]
    std::vector<int2> chunks;             // (row, x0)
    std::vector<uint32_t> mask;           // [nslots]
    std::vector<int32_t> slot_of_active;  // [n_active], active order = increasing box index
    std::vector<int64_t> box_of_active;   // [n_active]
};

// Returns "" on success, else a description of the inconsistency.
std::string build_index(const uint8_t *flags, int nx, int ny, int nz, int periodic, HostIndex &out);

}  // namespace lbm
