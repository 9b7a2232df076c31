// Totals of a caller-owned population array without any device allocation.
//
// Some callers cannot let this library allocate device memory: applications
// whose device memory is owned by their own pool and fixed budget, and
// latency-critical loops where cudaMalloc / cudaFree would synchronise the
// device.  lbm_totals_noalloc serves them: the caller passes the populations
// and the output buffer, and the per-block partial sums (the only scratch the
// reduction needs) live in a file-scope device array of fixed size instead of
// an allocation.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

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

// Host code cannot use g_noalloc_partials as an address: it stands for the
// device array, whose address cudaGetSymbolAddress gives per context.  The
// lookup is cached per device together with the identity of the context it
// was made in (cuCtxGetId), so that a context re-created after a
// cudaDeviceReset gets a fresh lookup instead of a stale address.  The cache
// is guarded by a mutex: host threads may call concurrently.
constexpr int MAX_DEVICES = 64;
struct ScratchAddress {
    unsigned long long ctx_id = 0;  // 0: not looked up yet
    double *ptr = nullptr;
};
std::mutex g_scratch_mu;
ScratchAddress g_scratch[MAX_DEVICES];

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points
// (the library links only the CUDA runtime).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
std::once_flag g_driver_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

void load_driver_entry_points() {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(fn);
}

// Identity of the calling thread's current context (0 if unavailable).
unsigned long long current_context_id() {
    std::call_once(g_driver_once, load_driver_entry_points);
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch in the current context of device dev.  The
// first call in a context looks it up (cudaGetSymbolAddress), which must not
// happen inside a stream capture: then LBM_ERR_STATE, nothing looked up.
lbm_status scratch_address(int dev, cudaStream_t st, double **out) {
    const unsigned long long id = current_context_id();
    if (id == 0) return LBM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchAddress &a = g_scratch[dev];
    if (a.ctx_id != id) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return LBM_ERR_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return LBM_ERR_STATE;
        double *p = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_partials) != cudaSuccess || !p)
            return LBM_ERR_CUDA;
        a.ptr = p;
        a.ctx_id = id;
    }
    *out = a.ptr;
    return LBM_OK;
}

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

template <int P>
cudaError_t launch_totals(const void *f, int64_t n, int64_t stride, float inv_s, double *partials, int nblocks,
                          double *out, cudaStream_t st) {
    // launched through cudaLaunchKernelEx, whose return value is this
    // launch's own status (an earlier, unrelated error of the caller stays
    // where it was)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3(NOALLOC_THREADS);
    cfg.stream = st;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_totals_contig<P>, f, n, stride, inv_s, partials);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(256);
    return cudaLaunchKernelEx(&cfg, k_totals_final, static_cast<const double *>(partials), nblocks, out);
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
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LBM_ERR_CUDA;
    // binds the device's primary context to this thread if no runtime call has yet
    if (cudaSetDevice(dev) != cudaSuccess) return LBM_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *partials = nullptr;
    const lbm_status ps = scratch_address(dev, st, &partials);
    if (ps != LBM_OK) return ps;
    const int64_t per_block = (int64_t)NOALLOC_THREADS * NOALLOC_CELLS_PER_THREAD;
    const int nblocks = (int)((n + per_block - 1) / per_block);
    const float inv_s = precision == LBM_FP16S ? 1.0f / s : 1.0f;
    cudaError_t e;
    if (precision == LBM_FP64)
        e = launch_totals<0>(f, n, stride, inv_s, partials, nblocks, out, st);
    else if (precision == LBM_FP32)
        e = launch_totals<1>(f, n, stride, inv_s, partials, nblocks, out, st);
    else
        e = launch_totals<2>(f, n, stride, inv_s, partials, nblocks, out, st);
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
