// lbm_noalloc.cu -- observables reduction that allocates nothing.
//
// lbm_observe keeps its block partial sums in the sim's device workspace.
// This file offers the same FP64 reduction to callers that cannot allocate
// device memory at the point where they need it: code that runs while a
// stream is being recorded into a graph, latency-critical loops where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable,
// and hosts whose device memory is entirely planned up front (a fixed HBM
// budget shared by many simulations).  Its scratch is a fixed array in the
// library's own device memory instead.
#include "lbm.h"
#include "lbm_internal.h"

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 16;
constexpr int kSums = 8;
// Scratch capacity: one row of 8 partial sums per block, 4096 blocks (256
// KiB), i.e. lattices of up to 4096 * 256 * 16 = 16,777,216 fluid nodes.
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxNodes = (long long)kMaxBlocks * kThreads * kNodesPerThread;
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_partials[kMaxBlocks * kSums];

lbm_status fail(lbm_status st, const char* fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return lbm_set_error(st, msg);  // reported by lbm_last_error()
}

std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};

// Device address of g_partials on the current device, looked up once per
// device.  In host code the name g_partials is only a host-side stand-in, so
// the kernels receive this address instead.
lbm_status partials_on_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess)
            return fail(LBM_ECUDA, "cudaGetSymbolAddress(scratch) on device %d: %s", dev,
                        cudaGetErrorString(e));
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return LBM_OK;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sums over the fluid nodes of fields [6][ny][nx]: sum phi, sum psi,
// sum phi x, sum phi y, sum phi u_x, sum phi u_y, non-finite count, node
// count; one row of partials per block (the grid grows with the lattice).
__global__ void __launch_bounds__(kThreads)
    noalloc_partial_kernel(const float* __restrict__ fld, int nx, int ny, int y0, int nfy,
                           double* __restrict__ part)
{
    double acc[kSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    const size_t N = (size_t)nx * ny;
    const long long total = (long long)nx * nfy;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = y0 + (int)(i / nx);
        const size_t o = (size_t)y * nx + x;
        const float phi = fld[o], ux = fld[N + o], uy = fld[2 * N + o], p = fld[3 * N + o];
        const float T = fld[4 * N + o], psi = fld[5 * N + o];
        const bool bad = !(isfinite(phi) && isfinite(ux) && isfinite(uy) && isfinite(p) &&
                           isfinite(T) && isfinite(psi));
        acc[0] += (double)phi;
        acc[1] += (double)psi;
        acc[2] += (double)phi * x;
        acc[3] += (double)phi * y;
        acc[4] += (double)phi * ux;
        acc[5] += (double)phi * uy;
        acc[6] += bad ? 1.0 : 0.0;
        acc[7] += 1.0;
    }
    __shared__ double sm[kThreads / 32][kSums];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSums; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sm[w][threadIdx.x];
        part[(size_t)blockIdx.x * kSums + threadIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kThreads)
    noalloc_final_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ out)
{
    __shared__ double sm[kThreads / 32][kSums];
    double acc[kSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < kSums; ++k) acc[k] += part[(size_t)b * kSums + k];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kSums; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sm[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

}  // namespace

extern "C" lbm_status lbm_reduce_observables_noalloc(const float* d_fields, int32_t nx, int32_t ny,
                                                      int32_t walls, double* d_sums, void* stream)
{
    if (!d_fields || !d_sums) return fail(LBM_EINVAL, "d_fields and d_sums must be device pointers");
    if (nx < 1 || ny < (walls ? 3 : 1) || (walls != 0 && walls != 1))
        return fail(LBM_EINVAL, "invalid lattice %dx%d (walls %d)", nx, ny, walls);
    const int nfy = walls ? ny - 2 : ny;
    const long long nodes = (long long)nx * nfy;
    if (nodes > kMaxNodes)
        return fail(LBM_EINVAL,
                    "lattice has %lld fluid nodes; the no-alloc reduction holds at most %lld "
                    "(%d blocks of %d threads x %d nodes)",
                    nodes, kMaxNodes, kMaxBlocks, kThreads, kNodesPerThread);
    if ((long long)nx * ny * 6 > (1LL << 31) - 1)
        return fail(LBM_EINVAL, "lattice %dx%d too large", nx, ny);
    double* part = nullptr;
    lbm_status st = partials_on_current_device(&part);
    if (st != LBM_OK) return st;
    const long long per_block = (long long)kThreads * kNodesPerThread;
    int nblocks = (int)((nodes + per_block - 1) / per_block);
    if (nblocks < 1) nblocks = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_partial_kernel<<<nblocks, kThreads, 0, s>>>(d_fields, nx, ny, walls ? 1 : 0, nfy, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ECUDA, "partial sums launch: %s", cudaGetErrorString(e));
    noalloc_final_kernel<<<1, kThreads, 0, s>>>(part, nblocks, d_sums);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LBM_ECUDA, "final sum launch: %s", cudaGetErrorString(e));
    return LBM_OK;
}
