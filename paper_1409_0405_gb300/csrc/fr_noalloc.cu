// fr_reduce_noalloc: the conserved-integral reduction for callers that
// cannot allocate device memory.
//
// The context-based fr_reduce keeps its per-block partial sums in a buffer
// that fr_create allocates.  Some callers cannot call cudaMalloc at all —
// for example code running under a memory pool or allocator that owns the
// whole device and forbids other allocations, or code on a path where an
// allocation (which may synchronise the device) is not allowed.  This
// variant takes plain device pointers for its input and output and keeps
// its scratch (one 7-double partial per block) in a file-scope static
// device array of fixed size, so it allocates nothing.
//
// Scratch: g_partials, FR_NOALLOC_MAX_BLOCKS x 7 doubles (229,376 bytes),
// resident on every GPU that loads this library until the process exits.
// Every call shares it and it keeps the last call's contents; each block
// overwrites its own slot before the final pass reads exactly the slots of
// the current call, so nothing needs clearing.  Calls that overlap on the
// GPU (different streams, or different host threads) race on it.
//
// Host code must not pass the array's name to a kernel: in host code it is
// only a stand-in for the device symbol.  The device address is obtained
// once per device with cudaGetSymbolAddress, with that device current, the
// first time the entry point is called on it; that first call should
// therefore come before any stream capture.  The cached address belongs to
// the device's primary context: after a cudaDeviceReset it would be stale,
// so a process that resets a device must not call this entry point again.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/fr.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPointsPerThread = 8;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[FR_NOALLOC_MAX_BLOCKS * 7];

// the limit documented in fr.h is the one enforced here
static_assert((int64_t)kThreads * kPointsPerThread * FR_NOALLOC_MAX_BLOCKS == FR_NOALLOC_MAX_POINTS,
              "FR_NOALLOC_MAX_POINTS must equal the blocks times the points per block");

double *g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__global__ void k_noalloc_partial(int64_t npts, int nu, const double *__restrict__ u,
                                  const double *__restrict__ wJ, double gamma, double *partial) {
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t base = (int64_t)blockIdx.x * kThreads * kPointsPerThread;
    for (int i = 0; i < kPointsPerThread; ++i) {
        const int64_t pt = base + (int64_t)i * kThreads + threadIdx.x;
        if (pt >= npts) break;
        const int64_t e = pt / nu, j = pt - e * nu;
        const double w = wJ[pt];
        double q[5];
        for (int v = 0; v < 5; ++v) {
            q[v] = u[(e * 5 + v) * nu + j];
            acc[v] += w * q[v];
        }
        const double ke = 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0];
        acc[5] += w * ke;
        const double p = (gamma - 1.0) * (q[4] - ke);
        bool bad = !(q[0] > 0.0) || !(p > 0.0);
        for (int v = 0; v < 5; ++v) bad = bad || !isfinite(q[v]);
        acc[6] += bad ? 1.0 : 0.0;
    }
    __shared__ double sh[7][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 7; ++k) {
        double x = acc[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double x = 0;
        for (int w = 0; w < kThreads / 32; ++w) x += sh[threadIdx.x][w];
        partial[(int64_t)blockIdx.x * 7 + threadIdx.x] = x;
    }
}

__global__ void k_noalloc_final(const double *partial, int nblocks, double *out) {
    if (threadIdx.x < 7) {
        double x = 0;
        for (int b = 0; b < nblocks; ++b) x += partial[(int64_t)b * 7 + threadIdx.x];
        out[threadIdx.x] = x;
    }
}

}  // namespace

extern "C" int fr_reduce_noalloc(int64_t ne, int nu, const double *u_dev, const double *wJ_dev, double gamma,
                                 double *out_dev, void *cuda_stream) {
    if (ne < 0 || nu <= 0 || !u_dev || !wJ_dev || !out_dev || !(gamma > 1.0)) return FR_ERR_ARG;
    // bound ne before forming ne * nu, which could otherwise overflow
    if (ne > FR_NOALLOC_MAX_POINTS / nu) return FR_ERR_ARG;
    const int64_t npts = ne * (int64_t)nu;
    const int64_t per_block = (int64_t)kThreads * kPointsPerThread;
    const int64_t nblocks = (npts + per_block - 1) / per_block;
    if (nblocks > FR_NOALLOC_MAX_BLOCKS) return FR_ERR_ARG;  // npts > FR_NOALLOC_MAX_POINTS
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FR_ERR_CUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return FR_ERR_CUDA;
            }
            g_partials_addr[dev] = (double *)p;
        }
        scratch = g_partials_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (nblocks > 0) k_noalloc_partial<<<(unsigned)nblocks, kThreads, 0, s>>>(npts, nu, u_dev, wJ_dev, gamma, scratch);
    k_noalloc_final<<<1, 32, 0, s>>>(scratch, (int)nblocks, out_dev);
    return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ERR_CUDA;
}
