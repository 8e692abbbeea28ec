// Host helpers shared by the single-lattice and batch parts of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_internal.h"

constexpr int kMaxTileThreadsHost = 512;

// Workspace layout of one lattice (byte offsets, 256-byte aligned).
struct Plan {
    int64_t N = 0;
    int two = 1;                 // two-lattice algorithm
    int halo_grid = 0;           // one-lattice algorithm with a buffer grid (NPOL, NSOL)
    int tx = 0, ty = 1, ntx = 0, nty = 0;
    size_t pop[2] = {0, 0};
    size_t halo = 0;
    int64_t halo_parity_elems = 0;
    size_t links = 0, mom = 0, mom_bytes = 0, partials = 0, misc = 0, total = 0;
};

// One lattice: parameters, workspace plan, kernel arguments, scheduling state.
struct lbm_lattice {
    lbm_params p;
    Plan pl;
    lbm::HostArgs h;
    const lbm::Ops *ops;
    cudaStream_t stream;
    cudaStream_t cap;
    char *ws;
    int cur;            // current lattice (two-lattice algorithms)
    int64_t steps;      // updates since lbm_init
    int64_t fluid;
    double *partials;
    double *red_out;
    unsigned int *err;
    unsigned long long *count;
    cudaGraphExec_t graph[4];
    int graph_steps;
    char *stage;                // page-locked read-back staging (lazy), two chunks
    cudaEvent_t stage_ev[2];
};

lbm_status lbm_fail(lbm_status s, const char *fmt, ...);
// Tensor map (TMA descriptor) of an FP32 tensor of `rank` dimensions (dims
// innermost first, byte strides of dimensions 1 .. rank-1, copy box); false
// when the CUDA driver's encoder is unavailable or rejects the description.
bool lbm_encode_f32_tensor_map(lbm::TmaDesc *out, int rank, void *base, const uint64_t *dims,
                               const uint64_t *strides, const uint32_t *box);
lbm_status lbm_cuda_fail(cudaError_t e, const char *where);
lbm_status lbm_check_params(const lbm_params *p);
lbm_status lbm_plan(const lbm_params *p, Plan *pl);
const lbm::Ops *ops_for_storage(int storage);
void lbm_fill_args(const lbm_params *p, const Plan &pl, char *ws, const lbm::Ops *ops, lbm::HostArgs *h);
int64_t layout_addr(int layout, int64_t N, int64_t n, int i);
lbm_status lbm_pops_to_host(const unsigned char *raw, int storage, int layout, int rev, int64_t N,
                            void *host, int32_t as);
