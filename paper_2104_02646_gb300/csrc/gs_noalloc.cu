// gs_loss_noalloc: the position loss L = sum_i |x_i - x*_i|^2 (FP64) and its
// seed dL/dx = 2 (x - x*), computed without any device allocation.
//
// Who needs it: callers that cannot allocate device memory while they run.
// A real-time control loop (for example a model-predictive controller that
// evaluates this loss every control tick) cannot afford cudaMalloc, which may
// synchronise the device and take unbounded time; a host application that
// owns a fixed memory pool may forbid libraries from allocating at all.  The
// regular path (gs_rollout with a target) allocates its reduction scratch
// through the context; this entry point instead uses one fixed scratch array
// that lives in this library's device memory.
//
// The scratch is a file-scope __device__ array of GS_NOALLOC_MAX_NODES / 256
// doubles (128 KiB): one FP64 partial sum per 256-node block.  Every GPU that
// loads the library holds it until the process exits.  All calls share it and
// it keeps the last call's contents; each call overwrites every partial it
// reads, so nothing has to start at zero, but calls whose work overlaps on the
// GPU (different streams, or different host threads on one device) race on
// the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = GS_NOALLOC_MAX_NODES / kThreads;

static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks];

// Per-device address of the scratch array.  In host code the array's name is
// only a host-side stand-in, so the device address is looked up once per
// device (with that device current) and passed to the kernels.  The cached
// address belongs to the device's primary context: a cudaDeviceReset by the
// host application destroys it, and the entry point is not to be used on
// that device afterwards.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

gs_status scratch_address(double** out) {
    int dev = 0;
    GS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(GS_EUNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return GS_OK;
}

// one FP64 partial per block of 256 nodes (fixed-order tree), and the seed
__global__ void k_noalloc_partials(const float* __restrict__ x, const float* __restrict__ target, int n,
                                   double* __restrict__ partials, float* __restrict__ dLdx) {
    __shared__ double red[kThreads];
    const int i = blockIdx.x * kThreads + threadIdx.x;
    double acc = 0.0;
    if (i < n) {
        for (int k = 0; k < 3; ++k) {
            const double d = (double)x[3 * i + k] - (double)target[3 * i + k];
            acc += d * d;
            if (dLdx) dLdx[3 * i + k] = (float)(2.0 * d);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// sum of the partials in block order
__global__ void k_noalloc_finalize(const double* __restrict__ partials, int nblocks, double* out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b];
        *out = s;
    }
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_loss_noalloc(const float* x, const float* target, int n_nodes, double* loss_out,
                                     float* dL_dx, void* stream) try {
    clear_error();
    if (!x || !target || !loss_out) return set_error(GS_EINVAL, "gs_loss_noalloc: x, target and loss_out are required");
    if (n_nodes < 0) return set_error(GS_EINVAL, "gs_loss_noalloc: n_nodes must be >= 0");
    if (n_nodes > GS_NOALLOC_MAX_NODES)
        return set_error(GS_EINVAL, "gs_loss_noalloc: n_nodes " + std::to_string(n_nodes) +
                                        " exceeds the fixed scratch limit GS_NOALLOC_MAX_NODES = " +
                                        std::to_string(GS_NOALLOC_MAX_NODES));
    double* scratch = nullptr;
    GS_TRY(scratch_address(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (n_nodes + kThreads - 1) / kThreads;
    if (nblocks > 0) k_noalloc_partials<<<nblocks, kThreads, 0, s>>>(x, target, n_nodes, scratch, dL_dx);
    k_noalloc_finalize<<<1, 32, 0, s>>>(scratch, nblocks, loss_out);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
} GS_ABI_CATCH
