// Totals of a caller-owned population array without any device allocation.
//
// Some callers cannot let this library allocate device memory: applications
// whose device memory is owned by their own pool and fixed budget, and
// latency-critical loops where cudaMalloc / cudaFree would synchronise the
// device.  lbm_totals_noalloc serves them: the caller passes the populations
// and the output buffer, and the per-block partial sums (the only scratch the
// reduction needs) live in a file-scope device array of fixed size instead of
// an allocation.
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace {

// Cells reduced by one block; blocks are limited by the static scratch.
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_CELLS_PER_THREAD = 16;
constexpr int NOALLOC_MAX_BLOCKS = 4096;
static_assert((int64_t)NOALLOC_MAX_BLOCKS * NOALLOC_THREADS * NOALLOC_CELLS_PER_THREAD == LBM_NOALLOC_MAX_CELLS,
              "header limit and scratch size disagree");

// Scratch: one 8-double partial per block (256 KB).  Every device that loads
// the library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * lbm::REDUCE_SLOTS];

// Device addresses of g_noalloc_partials, looked up once per device.
int g_scratch_ready[64];
double *g_scratch_ptr[64];

template <int P>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    k_totals_contig(const void *f, int64_t n, int64_t stride, float inv_scale, double *partials) {
    double hv[6] = {0, 0, 0, 0, 0, 0};
    const int64_t first = (int64_t)blockIdx.x * NOALLOC_THREADS * NOALLOC_CELLS_PER_THREAD + threadIdx.x;
    for (int k = 0; k < NOALLOC_CELLS_PER_THREAD; ++k) {
        const int64_t cell = first + (int64_t)k * NOALLOC_THREADS;
        if (cell >= n) break;
        double d[27], rho, ux, uy, uz, v[6];
        lbm::load_cell<P>(f, stride, (int)cell, inv_scale, d);
        lbm::moments_of(d, rho, ux, uy, uz);
        lbm::health_values(rho, ux, uy, uz, v);
        for (int q = 0; q < 6; ++q) hv[q] = (q == 4) ? fmax(hv[q], v[q]) : hv[q] + v[q];
    }
    lbm::block_reduce_write(hv, partials);
}

// Fixed-order sum of the partials (one block): out = mass, momentum (3),
// max |u|, non-finite count.
__global__ void __launch_bounds__(256) k_totals_final(const double *partials, int nblocks, double *out) {
    __shared__ double sh[256][6];
    double r[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += 256)
        for (int q = 0; q < 6; ++q) {
            const double v = partials[(size_t)b * lbm::REDUCE_SLOTS + q];
            r[q] = (q == 4) ? fmax(r[q], v) : r[q] + v;
        }
    for (int q = 0; q < 6; ++q) sh[threadIdx.x][q] = r[q];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < 6; ++q)
                sh[threadIdx.x][q] = (q == 4) ? fmax(sh[threadIdx.x][q], sh[threadIdx.x + h][q])
                                              : sh[threadIdx.x][q] + sh[threadIdx.x + h][q];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) out[q] = sh[0][q];
}

}  // namespace

extern "C" lbm_status lbm_totals_noalloc(const void *f, int32_t precision, float fp16_scale, int64_t n, int64_t stride,
                                         double *out, void *stream) {
    if (!f || !out || n < 1 || stride < n) return LBM_ERR_ARG;
    if (n > LBM_NOALLOC_MAX_CELLS) return LBM_ERR_ARG;  // beyond the static scratch
    if (stride > (int64_t)INT32_MAX) return LBM_ERR_ARG;
    if (precision < LBM_FP64 || precision > LBM_FP16S) return LBM_ERR_ARG;
    const float s = fp16_scale == 0.0f ? 4096.0f : fp16_scale;
    if (!(s > 0.0f)) return LBM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LBM_ERR_CUDA;
    if (!g_scratch_ready[dev]) {  // set-up on this device's first call
        double *p = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ready[dev] = 1;
    }
    double *partials = g_scratch_ptr[dev];
    const int64_t per_block = (int64_t)NOALLOC_THREADS * NOALLOC_CELLS_PER_THREAD;
    const int nblocks = (int)((n + per_block - 1) / per_block);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float inv_s = precision == LBM_FP16S ? 1.0f / s : 1.0f;
    if (precision == LBM_FP64)
        k_totals_contig<0><<<nblocks, NOALLOC_THREADS, 0, st>>>(f, n, stride, inv_s, partials);
    else if (precision == LBM_FP32)
        k_totals_contig<1><<<nblocks, NOALLOC_THREADS, 0, st>>>(f, n, stride, inv_s, partials);
    else
        k_totals_contig<2><<<nblocks, NOALLOC_THREADS, 0, st>>>(f, n, stride, inv_s, partials);
    k_totals_final<<<1, 256, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
