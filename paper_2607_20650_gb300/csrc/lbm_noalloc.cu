// Total-mass reduction that needs no device allocation and no workspace.
//
// Some callers cannot hand this library any device memory of their own: a
// host application whose framework owns every device allocation through its
// own pool and forbids direct cudaMalloc, or a control loop that must not
// pay the implicit synchronisation and latency of an allocation while it
// runs. lbm_mass_f32_noalloc serves them: its only scratch (one FP64 partial
// sum per block of nodes, plus the final sum) lives in a fixed file-scope
// device array that is part of the loaded library, so the call itself never
// allocates. The caller passes inputs and receives the output.
//
// Limits and sharing rules:
//  - at most kMaxBlocks blocks of kNodesPerBlock nodes: N <= 134,217,728;
//  - the array is one per GPU that loads the library and is held until the
//    process exits;
//  - every call reuses the same array, so calls whose GPU work overlaps (on
//    different streams, or from different host threads) race on it;
//  - every block overwrites its own partial and the final kernel overwrites
//    the sum, so nothing has to be cleared between calls;
//  - the first call on a device does the set-up: it looks up the array's
//    device address (cudaGetSymbolAddress) with that device current and keeps
//    it for the process; make that first call before any stream capture;
//  - the kept address is not refreshed after cudaDeviceReset, so the entry
//    point must not be called after a reset of the device in this process;
//  - every call copies the result into host memory and synchronises its
//    stream before returning.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "lbm.h"
#include "lbm_capi_internal.h"

namespace {

constexpr int kNodesPerBlock = 2048;
constexpr int kThreads = 256;
constexpr int64_t kMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

// Block partials [0, kMaxBlocks) and the final sum at [kMaxBlocks].
__device__ __align__(256) double g_mass_scratch[kMaxBlocks + 32];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};

// The same quantity as the workspace reduction (over fluid nodes,
// rho = 1 + sum_i h_i with h in canonical order h[i*N + n], in FP64) in a
// different fixed order: blocks of kNodesPerBlock nodes, then the block sums
// in index order. It agrees with lbm_mass to round-off, and repeated calls
// on the same data give identical bits.
__global__ void __launch_bounds__(kThreads) k_mass_blocks(const float *h, const uint8_t *solid,
                                                          uint32_t N, double *partials) {
    __shared__ double red[kThreads];
    const uint32_t n0 = blockIdx.x * (uint32_t)kNodesPerBlock;
    double acc = 0.0;
    for (uint32_t k = threadIdx.x; k < (uint32_t)kNodesPerBlock; k += kThreads) {
        const uint32_t n = n0 + k;
        if (n >= N || solid[n]) continue;
        double r = 1.0;
        for (int i = 0; i < 9; ++i) r += (double)h[(uint64_t)i * N + n];
        acc += r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_mass_total(const double *partials, int nblocks, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[b];
    *out = s;
}

// Device address of g_mass_scratch on the current device (looked up once).
lbm_status scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return lbm_fail(LBM_EUNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaGetSymbolAddress(g_mass_scratch)");
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_mass_f32_noalloc(const float *d_h, const uint8_t *d_solid, int64_t N,
                                           double *out, void *cuda_stream) {
    if (!d_h || !d_solid || !out) return lbm_fail(LBM_EINVAL, "lbm_mass_f32_noalloc: NULL argument");
    if (N < 1) return lbm_fail(LBM_EINVAL, "lbm_mass_f32_noalloc: N must be >= 1");
    const int64_t nblocks = (N + kNodesPerBlock - 1) / kNodesPerBlock;
    if (nblocks > kMaxBlocks)
        return lbm_fail(LBM_EINVAL,
                        "lbm_mass_f32_noalloc: N = %lld exceeds the fixed scratch (at most %lld nodes)",
                        (long long)N, (long long)(kMaxBlocks * kNodesPerBlock));
    double *scratch = nullptr;
    lbm_status s = scratch_for_current_device(&scratch);
    if (s != LBM_OK) return s;
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    k_mass_blocks<<<(unsigned)nblocks, kThreads, 0, st>>>(d_h, d_solid, (uint32_t)N, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lbm_cuda_fail(e, "k_mass_blocks");
    k_mass_total<<<1, 32, 0, st>>>(scratch, (int)nblocks, scratch + kMaxBlocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return lbm_cuda_fail(e, "k_mass_total");
    e = cudaMemcpyAsync(out, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaStreamSynchronize");
    return LBM_OK;
}
