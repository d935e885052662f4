// dc_eval_points_noalloc: the FP64 direct-sum evaluation of dc_eval_points
// for callers that cannot allocate device memory while they run -- for
// example code inside a render loop whose allocator belongs to another
// framework, code running under a memory budget that forbids growth, or a
// thread that must not take the allocator's locks.  All scratch lives in a
// fixed file-scope device array instead of context-owned cudaMalloc memory.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "dc_internal.h"

namespace dc {

namespace {

// Segment densities of one call: [kNoAllocMaxSegments][3] sigma_bar followed
// by [kNoAllocMaxSegments][3] mu_bar (12 MiB of FP64), held by every GPU
// that loads the library until the process exits.
constexpr int kNoAllocMaxSegments = 1 << 18;
static __device__ __align__(256) double g_noalloc_seg[2 * 3 * (size_t)kNoAllocMaxSegments];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current (the caller has checked that the
// current device is the context's).  The cached address belongs to the
// device's primary context: it does not survive a cudaDeviceReset, after
// which every context of the library must be rebuilt anyway.
cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_seg);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

int noalloc_max_segments() { return kNoAllocMaxSegments; }

// sigma and mu at the nodes -> segment values in the static scratch, then
// the direct sum at the points; no allocation of any kind.
cudaError_t eval_points_noalloc(const DevGeom &G, const double *sigma, const double *mu,
                                const double *xy, int n, double *out, cudaStream_t st,
                                std::string &err) {
    if (G.S > kNoAllocMaxSegments) {
        err = "eval_points_noalloc: the drawing has " + std::to_string(G.S) +
              " segments; the no-allocation path holds at most " +
              std::to_string(kNoAllocMaxSegments);
        return cudaErrorInvalidValue;
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        err = std::string("eval_points_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return e;
    }
    double *sbar = scratch, *mbar = scratch + 3 * (size_t)kNoAllocMaxSegments;
    // every scratch entry read below is written here first: nothing to clear
    if ((e = launch_interp(G, sigma, sbar, st)) != cudaSuccess) return e;
    if ((e = launch_interp(G, mu, mbar, st)) != cudaSuccess) return e;
    return launch_dense_eval_points(G, sbar, mbar, xy, n, out, st);
}

}  // namespace dc
