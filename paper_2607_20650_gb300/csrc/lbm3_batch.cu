// Batches of independent D3Q19 boxes behind the lbm3_batch_* calls of
// include/lbm.h: the batched form of the 2-D library carried to the 3-D
// kernels. Each case is a full box (lbm3_lattice) in its own region of the
// batch's workspace; one update of the batch is one launch over the packed
// (case, item) list, whose blocks run the single-box tile code on their
// case's arguments (k3_batch), captured into CUDA graphs of 64 updates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "lbm.h"
#include "lbm3_internal.h"
#include "lbm_capi_internal.h"
#include "lbm_internal.h"

#define CKB(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return lbm_cuda_fail(e_, #call);   \
    } while (0)

namespace {

constexpr int kGraph3Steps = 64;   // even: the parity after a graph is the one before
constexpr int kBatch3Nodes = 256;  // LPTL work item: consecutive nodes (and threads per block)

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct Batch3Layout {
    std::vector<Plan3> plans;
    std::vector<size_t> case_off;
    std::vector<int64_t> items;   // per case
    size_t case_bytes = 0, cases_off = 0, items_off = 0, misc_off = 0, total = 0;
    uint32_t nitems = 0;
};

lbm_status batch3_layout(int32_t ncases, const lbm3_params *params, Batch3Layout *bl) {
    if (ncases < 1) return lbm_fail(LBM_EINVAL, "lbm3 batch: ncases must be >= 1");
    if (!params) return lbm_fail(LBM_EINVAL, "lbm3 batch: params is NULL");
    const lbm3_params &p0 = params[0];
    bl->plans.resize(ncases);
    bl->items.resize(ncases);
    int64_t total_items = 0;
    for (int c = 0; c < ncases; ++c) {
        const lbm3_params &p = params[c];
        lbm_status s = lbm3_plan(&p, &bl->plans[c]);
        if (s != LBM_OK) return lbm_fail(s, "lbm3 batch case %d: %s", c, lbm_last_error());
        if (p.storage != p0.storage || p.layout != p0.layout || p.algo != p0.algo)
            return lbm_fail(LBM_EINVAL, "lbm3 batch case %d: storage, layout and algorithm must match case 0", c);
        if (p.algo == LBM_AA)
            return lbm_fail(LBM_EUNSUPPORTED, "lbm3 batch: the AA pattern runs on single boxes only");
        const Plan3 &pl = bl->plans[c], &pl0 = bl->plans[0];
        if (p.algo != LBM_LPTL && (pl.tx != pl0.tx || pl.ty != pl0.ty || pl.tz != pl0.tz))
            return lbm_fail(LBM_EINVAL, "lbm3 batch case %d: tile %dx%dx%d differs from case 0's %dx%dx%d", c,
                            pl.tx, pl.ty, pl.tz, pl0.tx, pl0.ty, pl0.tz);
        if (!lbm3_offsets_fit(&p, pl.N) || (p.flags & LBM_FLAG_WIDE_OFFSETS))
            return lbm_fail(LBM_EUNSUPPORTED, "lbm3 batch case %d: needs the 32-bit offset tables", c);
        bl->items[c] = p.algo == LBM_LPTL ? (pl.N + kBatch3Nodes - 1) / kBatch3Nodes
                                          : (int64_t)pl.ntx * pl.nty * pl.ntz;
        total_items += bl->items[c];
    }
    if (total_items >= ((int64_t)1 << 31)) return lbm_fail(LBM_EUNSUPPORTED, "lbm3 batch: too many work items");
    bl->nitems = (uint32_t)total_items;
    bl->case_bytes = ops3_for(p0.storage)->case_bytes;
    bl->cases_off = 0;
    bl->items_off = align256(bl->case_bytes * (size_t)ncases);
    bl->misc_off = bl->items_off + align256(2 * sizeof(uint32_t) * (size_t)total_items);
    size_t off = bl->misc_off + 256;
    bl->case_off.resize(ncases);
    for (int c = 0; c < ncases; ++c) {
        bl->case_off[c] = off;
        off += align256(bl->plans[c].total);
    }
    bl->total = off;
    return LBM_OK;
}

}  // namespace

struct lbm3_batch {
    int ncases;
    lbm3_params p0;
    const Ops3 *ops;
    Batch3Layout bl;
    std::vector<lbm3_lattice *> cases;
    char *ws;
    cudaStream_t stream, cap;
    unsigned int *err;
    long long *tctr;
    int cur;
    int64_t steps;
    cudaGraphExec_t graph[2];
};

extern "C" lbm_status lbm3_batch_workspace_bytes(int32_t ncases, const lbm3_params *params, size_t *bytes) {
    if (!bytes) return lbm_fail(LBM_EINVAL, "bytes is NULL");
    Batch3Layout bl;
    lbm_status s = batch3_layout(ncases, params, &bl);
    if (s == LBM_OK) *bytes = bl.total;
    return s;
}

extern "C" void lbm3_batch_destroy(lbm3_batch *B) {
    if (!B) return;
    cudaStreamSynchronize(B->stream);
    for (auto &g : B->graph)
        if (g) cudaGraphExecDestroy(g);
    for (auto *L : B->cases) lbm3_destroy(L);
    if (B->cap) cudaStreamDestroy(B->cap);
    delete B;
}

extern "C" lbm_status lbm3_batch_create(int32_t ncases, const lbm3_params *params, const uint8_t *const *masks,
                                        void *d_workspace, size_t bytes, void *cuda_stream, lbm3_batch **out) {
    if (!out) return lbm_fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!masks) return lbm_fail(LBM_EINVAL, "masks is NULL");
    if (!d_workspace || ((uintptr_t)d_workspace) % 256)
        return lbm_fail(LBM_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    lbm3_batch *B = new lbm3_batch();
    lbm_status s = batch3_layout(ncases, params, &B->bl);
    if (s != LBM_OK) {
        delete B;
        return s;
    }
    if (bytes < B->bl.total) {
        const size_t need = B->bl.total;
        delete B;
        return lbm_fail(LBM_ENOMEM, "lbm3 batch workspace too small: %zu given, %zu needed", bytes, need);
    }
    B->ncases = ncases;
    B->p0 = params[0];
    B->ops = ops3_for(params[0].storage);
    B->ws = (char *)d_workspace;
    B->stream = (cudaStream_t)cuda_stream;
    B->err = (unsigned int *)(B->ws + B->bl.misc_off);
    B->tctr = (long long *)(B->ws + B->bl.misc_off + 64);
    cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        B->cap = nullptr;
        lbm3_batch_destroy(B);
        return lbm_cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    std::vector<unsigned char> recs(B->bl.case_bytes * (size_t)ncases);
    std::vector<uint32_t> items;
    items.reserve(2 * (size_t)B->bl.nitems);
    for (int c = 0; c < ncases; ++c) {
        if (!masks[c]) {
            lbm3_batch_destroy(B);
            return lbm_fail(LBM_EINVAL, "lbm3 batch case %d: mask is NULL", c);
        }
        lbm3_lattice *L = nullptr;
        s = lbm3_create(&params[c], masks[c], B->ws + B->bl.case_off[c], B->bl.plans[c].total, cuda_stream, &L);
        if (s != LBM_OK) {
            lbm3_batch_destroy(B);
            return lbm_fail(s, "lbm3 batch case %d: %s", c, lbm_last_error());
        }
        B->cases.push_back(L);
        L->err = B->err;   // one divergence flag and one update counter for the batch
        L->tctr = B->tctr;
        B->ops->batch_case(L, recs.data() + (size_t)c * B->bl.case_bytes);
        for (int64_t t = 0; t < B->bl.items[c]; ++t) {
            items.push_back((uint32_t)c);
            items.push_back((uint32_t)t);
        }
    }
    e = cudaMemcpyAsync(B->ws + B->bl.cases_off, recs.data(), recs.size(), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->ws + B->bl.items_off, items.data(), items.size() * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->ws + B->bl.misc_off, 0, 256, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) {
        lbm3_batch_destroy(B);
        return lbm_cuda_fail(e, "lbm3 batch upload");
    }
    *out = B;
    return LBM_OK;
}

extern "C" lbm_status lbm3_batch_init(lbm3_batch *B, int32_t c, const double *rho, const double *ux,
                                      const double *uy, const double *uz) {
    if (!B || c < 0 || c >= B->ncases) return lbm_fail(LBM_EINVAL, "lbm3_batch_init: bad batch or case");
    if (B->steps != 0) return lbm_fail(LBM_EINVAL, "lbm3_batch_init: only before the first lbm3_batch_step");
    return lbm3_init(B->cases[c], rho, ux, uy, uz);
}

static cudaError_t batch3_block(lbm3_batch *B, cudaStream_t st, int64_t count, int want_moments) {
    Batch3Launch b;
    b.layout = B->p0.layout;
    b.algo = B->p0.algo;
    b.cases = B->ws + B->bl.cases_off;
    b.items = B->ws + B->bl.items_off;
    b.nitems = B->bl.nitems;
    b.tx = B->bl.plans[0].tx;
    b.ty = B->bl.plans[0].ty;
    b.tz = B->bl.plans[0].tz;
    b.block_1d = kBatch3Nodes;
    int cur = B->cur;
    for (int64_t k = 0; k < count; ++k) {
        b.src = cur;
        b.toff = (int)k;
        b.mom = (want_moments && k == count - 1) ? 1 : 0;
        cudaError_t e = B->ops->batch_step(b, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return lbm::launch_bump_counter(B->tctr, count, st);
}

extern "C" lbm_status lbm3_batch_step(lbm3_batch *B, int64_t nsteps, uint32_t want_moments) {
    if (!B) return lbm_fail(LBM_EINVAL, "batch is NULL");
    if (nsteps < 0) return lbm_fail(LBM_EINVAL, "nsteps must be >= 0");
    int64_t left = nsteps;
    while (left > kGraph3Steps || (left == kGraph3Steps && !want_moments)) {
        cudaGraphExec_t &ex = B->graph[B->cur];
        if (!ex) {
            cudaGraph_t g = nullptr;
            CKB(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = batch3_block(B, B->cap, kGraph3Steps, 0);
            cudaError_t e2 = cudaStreamEndCapture(B->cap, &g);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return lbm_cuda_fail(e, "capturing D3Q19 batch updates");
            }
            if (e2 != cudaSuccess) return lbm_cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return lbm_cuda_fail(e, "cudaGraphInstantiate");
        }
        CKB(cudaGraphLaunch(ex, B->stream));
        B->steps += kGraph3Steps;
        left -= kGraph3Steps;
    }
    if (left > 0) {
        CKB(batch3_block(B, B->stream, left, want_moments ? 1 : 0));
        if (left & 1) B->cur ^= 1;
        B->steps += left;
    }
    for (auto *L : B->cases) {
        L->cur = B->cur;
        L->steps = B->steps;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm3_batch_sync(lbm3_batch *B) {
    if (!B) return lbm_fail(LBM_EINVAL, "batch is NULL");
    CKB(cudaStreamSynchronize(B->stream));
    return lbm3_check(B->cases[0]);   // every case shares the batch's flag
}

extern "C" lbm_status lbm3_batch_read_moments(lbm3_batch *B, int32_t c, double *rho, double *ux, double *uy,
                                              double *uz) {
    if (!B || c < 0 || c >= B->ncases) return lbm_fail(LBM_EINVAL, "bad batch or case");
    return lbm3_read_moments(B->cases[c], rho, ux, uy, uz);
}

extern "C" lbm_status lbm3_batch_read_populations(lbm3_batch *B, int32_t c, void *host, int32_t as) {
    if (!B || c < 0 || c >= B->ncases) return lbm_fail(LBM_EINVAL, "bad batch or case");
    return lbm3_read_populations(B->cases[c], host, as);
}

extern "C" lbm_status lbm3_batch_mass(lbm3_batch *B, int32_t c, double *out) {
    if (!B || c < 0 || c >= B->ncases) return lbm_fail(LBM_EINVAL, "bad batch or case");
    return lbm3_mass(B->cases[c], out);
}

extern "C" lbm_status lbm3_batch_get_info(lbm3_batch *B, int64_t *items, int64_t *cells, int64_t *fluid_cells,
                                          double *bytes_per_update) {
    if (!B) return lbm_fail(LBM_EINVAL, "batch is NULL");
    int64_t n = 0, f = 0;
    double by = 0.0;
    for (auto *L : B->cases) {
        lbm_info info;
        lbm_status s = lbm3_get_info(L, &info);
        if (s != LBM_OK) return s;
        n += info.cells;
        f += info.fluid_cells;
        by += info.bytes_per_update;
    }
    if (items) *items = B->bl.nitems;
    if (cells) *cells = n;
    if (fluid_cells) *fluid_cells = f;
    if (bytes_per_update) *bytes_per_update = by;
    return LBM_OK;
}
