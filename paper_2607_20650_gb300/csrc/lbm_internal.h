// Host-side interface between the C ABI (lbm_capi.cu) and the kernel
// translation units (one per storage type). No device types appear here.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

// An opaque tensor-map descriptor for the tensor copies (the 128-byte,
// 64-byte aligned object the CUDA driver encodes), passed to kernels by value.
struct alignas(64) TmaDesc {
    unsigned char bytes[128];
};

// Everything a kernel launch needs, in host types.
struct HostArgs {
    int nx, ny;
    int64_t N;
    int bw, be, bs, bn;
    int layout, algo, storage, rounding;
    double omega, kf, fx, fy, ux_in, uy_in, rho_out;
    uint64_t seed;
    int tile_x, tile_y, ntx, nty;
    int block_1d;              // LPTL block size
    uint32_t flags;            // lbm_params.flags
    uint64_t nx_magic;         // ceil(2^64 / nx) for n -> (x, y); 0 when nx == 1
    uint32_t pf;               // L2 prefetch distance: nodes (LPTL) or rows (NPTL); 0 = off
    const uint8_t *links;
    void *pop[2];              // pop[1] == nullptr for one-lattice algorithms
    void *halo;                // one-lattice buffer grid (2 parities)
    int64_t halo_parity_elems; // elements per parity
    void *mom;                 // 3N compute-type values
    unsigned int *err;
    long long *tctr;           // device update counter (stochastic rounding keys)
    int tma;                   // NSOL, FP32: the tile is staged by one tensor copy (tmap)
    TmaDesc tmap;
};

// One update: which lattice is the source, the halo parity that is read,
// offset added to the device update counter, and whether moments are stored.
struct StepCall {
    int src;
    int rd_parity;
    int toff;
    int want_moments;
};

struct Ops {
    cudaError_t (*step)(const HostArgs &, const StepCall &, cudaStream_t);
    // Equilibrium from FP64 rho/ux/uy (device, count nodes from n0; NULL -> 1/0).
    cudaError_t (*init)(const HostArgs &, const double *rho, const double *ux, const double *uy,
                        int64_t n0, int64_t count, cudaStream_t);
    // Copy tile-edge populations of lattice `src` into halo parity `parity`.
    cudaError_t (*publish)(const HostArgs &, int src, int parity, cudaStream_t);
    // Store h = 0 at every solid node of lattice `src`.
    cudaError_t (*zero_solid)(const HostArgs &, int src, cudaStream_t);
    // rho = 1 + sum h, v = sum h c (- F/2 if post_collision) into mom.
    cudaError_t (*state_moments)(const HostArgs &, int src, int post_collision, cudaStream_t);
    // FP64 block partial sums: mass (1 value) or force (2 values) per block.
    cudaError_t (*mass)(const HostArgs &, int src, double *partials, int nblocks, cudaStream_t);
    cudaError_t (*force)(const HostArgs &, int src, const uint8_t *body, double *partials,
                         int nblocks, cudaStream_t);
    // Moments buffer (compute type) -> FP32 device arrays.
    cudaError_t (*moments_f32)(const HostArgs &, float *r, float *u, float *v, cudaStream_t);
    int (*lptl_block)(int layout);  // occupancy-chosen LPTL block size
    void (*prepare)();              // one-time kernel attributes (called at create)
    // Batches: one persistent launch over the packed tile list.
    // kind = layout * 4 + algo shared by every case, or -1 for a mixed batch.
    cudaError_t (*batch_step)(int kind, const void *cases, const void *tiles, uint32_t ntiles, int grid,
                              int cur, int toff, int want_moments, cudaStream_t);
    int (*batch_grid)(int kind);                           // resident blocks on the device
    void (*batch_case)(const HostArgs &, void *out);       // device record of one case
    size_t batch_case_bytes;
    size_t elem;               // bytes per stored population
    size_t compute;            // bytes per compute value
};

const Ops &ops_f64();
const Ops &ops_f32();
const Ops &ops_f16();
const Ops &ops_bf16();

// Shared kernels (lbm_common.cu).
cudaError_t launch_links(int nx, int ny, int bw, int be, int bs, int bn, const uint8_t *mask,
                         uint8_t *links, cudaStream_t);
cudaError_t launch_count_fluid(const uint8_t *links, int64_t N, unsigned long long *out,
                               cudaStream_t);
cudaError_t launch_sum_partials(const double *partials, int nblocks, int width, double *out,
                                cudaStream_t);
cudaError_t launch_bump_counter(long long *ctr, long long by, cudaStream_t);
cudaError_t launch_quantize(int storage, int rounding, uint64_t seed, int64_t t, const float *in,
                            void *out, float *back, int64_t count, cudaStream_t);

constexpr int kReduceBlocks = 1024;
constexpr int kReduceThreads = 256;
constexpr int kBatchTileNodes = 256;  // threads per batch block = nodes per LPTL tile
constexpr int kBatchSuperHost = 4;    // tiles per work item of a two-lattice case

}  // namespace lbm
