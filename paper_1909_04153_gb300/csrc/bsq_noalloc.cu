// bsq_noalloc.cu -- the water volume sum(max(w - b, 0)) dx dy of caller-owned
// device arrays, computed without allocating any memory.
//
// The regular path (bsq_info) reduces the depth into per-block partial sums
// held in a buffer that bsq_create allocated.  Here the partial sums (one per
// grid row) live in a fixed file-scope device array instead, so a caller that
// owns all of its device memory can use the reduction without the library
// ever calling cudaMalloc.  The array holds BSQ_NOALLOC_MAX_ROWS doubles
// (128 KiB) on every device that loads the library, until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/bsq.h"

namespace {

// One partial sum per row.  Each call writes every entry it later reads, so
// nothing has to be cleared between calls; the array keeps the last call's
// values.
static __device__ __align__(256) double g_row_sums[BSQ_NOALLOC_MAX_ROWS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_row_sums_addr[kMaxDevices] = {nullptr};

// Row j: sum over i of max(w - b, 0), one warp per row, in double.
template <typename T>
__global__ void __launch_bounds__(256) k_depth_row_sums(const T *w, const T *b, int nx, int ny, long long pitch,
                                                        double *rows)
{
    const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= ny) return;
    const T *wr = w + (long long)warp * pitch, *br = b + (long long)warp * pitch;
    double s = 0.0;
    for (int i = lane; i < nx; i += 32) {
        T h = wr[i] - br[i];
        s += h > (T)0 ? (double)h : 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rows[warp] = s;
}

// Sum of the row sums in a fixed order (deterministic), times dx dy.
__global__ void __launch_bounds__(256) k_sum_rows(const double *rows, int ny, double dxdy, double *out)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int j = threadIdx.x; j < ny; j += 256) s += rows[j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * dxdy;
}

// Device address of g_row_sums for the current device, looked up on the first
// call made with that device current.
bsq_status row_sums_address(double **ptr)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSQ_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return BSQ_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_row_sums_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_row_sums) != cudaSuccess || !p) return BSQ_ERR_CUDA;
        g_row_sums_addr[dev] = (double *)p;
    }
    *ptr = g_row_sums_addr[dev];
    return BSQ_OK;
}

}  // namespace

extern "C" bsq_status bsq_mass_noalloc(int precision, const void *w_dev, const void *b_dev, int nx, int ny,
                                       long long pitch, double dx, double dy, double *mass_dev,
                                       void *cuda_stream)
{
    if (!w_dev || !b_dev || !mass_dev || nx < 1 || ny < 1 || pitch < nx || !(dx > 0) || !(dy > 0))
        return BSQ_ERR_ARG;
    if (precision != BSQ_FP32 && precision != BSQ_FP64) return BSQ_ERR_ARG;
    if (ny > BSQ_NOALLOC_MAX_ROWS) return BSQ_ERR_ARG;  // more rows than the static array holds
    cudaGetLastError();  // an earlier failed launch elsewhere must not be reported as this call's
    double *rows = nullptr;
    bsq_status st = row_sums_address(&rows);
    if (st != BSQ_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = (int)(((long long)ny * 32 + 255) / 256);
    if (precision == BSQ_FP64)
        k_depth_row_sums<double><<<blocks, 256, 0, s>>>((const double *)w_dev, (const double *)b_dev, nx, ny,
                                                        pitch, rows);
    else
        k_depth_row_sums<float><<<blocks, 256, 0, s>>>((const float *)w_dev, (const float *)b_dev, nx, ny, pitch,
                                                       rows);
    k_sum_rows<<<1, 256, 0, s>>>(rows, ny, dx * dy, mass_dev);
    return cudaGetLastError() == cudaSuccess ? BSQ_OK : BSQ_ERR_CUDA;
}
