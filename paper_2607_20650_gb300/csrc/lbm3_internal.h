// Host-side interface between the D3Q19 C ABI (lbm3.cu, lbm3_batch.cu) and
// the D3Q19 kernel translation units (lbm3_ops_*.cu, one per storage type).
// No device types appear here.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm.h"

// Workspace layout of one box (byte offsets, 256-byte aligned).
struct Plan3 {
    int64_t N = 0;
    int tx = 0, ty = 1, tz = 1, ntx = 0, nty = 0, ntz = 0;
    size_t elem = 0, comp = 0;
    size_t pop[2] = {0, 0}, links = 0, mom = 0, mom_bytes = 0, partials = 0, misc = 0, total = 0;
    int one = 0;              // one lattice (AA pattern, NPOL, NSOL)
    size_t halo = 0;          // NPOL / NSOL buffer grid (two parities)
    int64_t halo_parity = 0;  // elements per parity
};

struct Ops3;

struct lbm3_lattice {
    lbm3_params p;
    Plan3 pl;
    const Ops3 *ops;
    char *ws;
    cudaStream_t stream, cap;
    int cur;
    int64_t steps;
    int64_t fluid;
    int block_1d;
    int off32;            // 32-bit offset tables usable (19 N and the pull shifts fit 31 bits)
    unsigned int *err;    // divergence flag (the box's own, or its batch's)
    long long *tctr;      // update counter: stochastic-rounding keys (the box's own, or its batch's)
    cudaGraphExec_t graph[2];
};

// One batched update: the case records and the work list in device memory.
struct Batch3Launch {
    int layout, algo;
    const void *cases;
    const void *items;    // (case, local item) pairs of uint32
    uint32_t nitems;
    int tx, ty, tz, block_1d;
    int src, toff, mom;
};

// Per-storage entry points (lbm3_ops_*.cu).
struct Ops3 {
    // One update: src = the update's parity (two lattices: the source lattice;
    // AA: the phase; NPOL/NSOL: the buffer-grid parity read).
    cudaError_t (*step)(const lbm3_lattice *L, cudaStream_t st, int src, int toff, int mom);
    // Equilibrium of `count` nodes from n0 from FP64 device arrays (NULL: 1 / 0) into lattice 0.
    cudaError_t (*init)(const lbm3_lattice *L, const double *const dv[4], uint32_t n0, uint32_t count,
                        cudaStream_t st);
    // rho, u of the stored state into the moments array.
    cudaError_t (*state_moments)(const lbm3_lattice *L, cudaStream_t st);
    // Fill buffer-grid parity `parity` from the stored state (NPOL, NSOL).
    cudaError_t (*publish)(const lbm3_lattice *L, int parity, cudaStream_t st);
    // FP64 block partial sums of the mass (one per block) and force (three).
    cudaError_t (*mass)(const lbm3_lattice *L, double *partials, cudaStream_t st);
    cudaError_t (*force)(const lbm3_lattice *L, const uint8_t *body, double *partials, cudaStream_t st);
    int (*block_1d)(int layout);   // occupancy-chosen LPTL block size
    void (*prepare)(int algo);     // one-time kernel attributes (NSOL shared memory)
    // Batches: the device record of one case, and one update of the batch.
    size_t case_bytes;
    void (*batch_case)(const lbm3_lattice *L, void *rec);
    cudaError_t (*batch_step)(const Batch3Launch &b, cudaStream_t st);
};

const Ops3 &ops3_f64();
const Ops3 &ops3_f32();
const Ops3 &ops3_f16();
const Ops3 &ops3_bf16();
const Ops3 *ops3_for(int storage);

inline size_t elem3_of(int storage) { return storage == LBM_F64 ? 8 : storage == LBM_F32 ? 4 : 2; }
inline size_t comp3_of(int storage) { return storage == LBM_F64 ? 8 : 4; }
inline bool inlet3_kind(int bc) { return bc == LBM_BC_INLET_EQ || bc == LBM_BC_INLET_ZOUHE; }
// Kind of the east x face: bc_x_east after an inlet west face, else bc_x.
inline int east3_kind(const lbm3_params *p) { return inlet3_kind(p->bc_x) ? p->bc_x_east : p->bc_x; }
// ceil(2^64 / d) for the division-free n -> (x, y, z); 0 for d <= 1.
inline uint64_t magic3(uint64_t d) { return d <= 1 ? 0ull : (~0ull / d) + 1ull; }

lbm_status lbm3_plan(const lbm3_params *p, Plan3 *pl);
bool lbm3_offsets_fit(const lbm3_params *p, int64_t N);
lbm_status lbm3_check(lbm3_lattice *L);
