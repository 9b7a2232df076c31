// Precision-independent kernels: the fixed-order final pass of the FP64
// health reduction and the time-average readback.
#include "lbm_internal.h"

namespace lbm {

int fluid_blocks(int32_t nchunks) {
    const int64_t threads = (int64_t)nchunks * CHUNK;
    return (int)((threads + STEP_THREADS - 1) / STEP_THREADS);
}

int node_blocks(int64_t n) { return (int)((n + STEP_THREADS - 1) / STEP_THREADS); }

// One block sums the per-block partials in a fixed order (each thread a
// fixed strided subset, then a fixed tree), so the totals are bitwise
// reproducible for a given lattice.  health: mass, momentum (3), max |u|,
// non-finite count.  A non-finite count > 0 raises bit 0 of *status.
__global__ void __launch_bounds__(256) k_finalize(const double *partials, int nblocks, double *health,
                                                  uint32_t *status) {
    __shared__ double sh[256][6];
    double r[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += 256) {
        const double *p = partials + (size_t)b * REDUCE_SLOTS;
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = (k == 4) ? fmax(r[k], p[k]) : r[k] + p[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] = r[k];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
#pragma unroll
            for (int k = 0; k < 6; ++k)
                sh[threadIdx.x][k] = (k == 4) ? fmax(sh[threadIdx.x][k], sh[threadIdx.x + h][k])
                                              : sh[threadIdx.x][k] + sh[threadIdx.x + h][k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) health[k] = sh[0][k];
        if (sh[0][5] > 0.0) *status |= 1u;
    }
}

cudaError_t launch_finalize(const double *partials, int nblocks, double *health, uint32_t *status,
                            cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(partials, nblocks, health, status);
    return cudaGetLastError();
}

__global__ void k_stats_mean(const double *stats, int ncomp, const int32_t *slot_of_active, int64_t n, int64_t stride,
                             double inv_n, double *out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int slot = slot_of_active[k];
    for (int q = 0; q < ncomp; ++q) out[(size_t)ncomp * k + q] = stats[(size_t)q * stride + slot] * inv_n;
}

cudaError_t launch_stats_mean(const double *stats, int ncomp, const int32_t *slot_of_active, int64_t n, int64_t stride,
                              double inv_n, double *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_stats_mean<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(stats, ncomp, slot_of_active, n, stride, inv_n, out);
    return cudaGetLastError();
}

// Split per-cell moments (rho, ux, uy, uz) in active order into rho[n] and
// u[n][3], so that both go to the caller's host arrays in one copy each.
__global__ void k_split_moments(const double *in, int64_t n, double *rho, double *u) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    rho[k] = in[4 * k];
    u[3 * k] = in[4 * k + 1];
    u[3 * k + 1] = in[4 * k + 2];
    u[3 * k + 2] = in[4 * k + 3];
}

cudaError_t launch_split_moments(const double *in, int64_t n, double *rho, double *u, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_split_moments<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, n, rho, u);
    return cudaGetLastError();
}

}  // namespace lbm
